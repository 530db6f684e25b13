// bvh_build.cpp -- host construction of the closest-point BVH (Sec. 4
// "Setup": walk on spheres answers its closest-point queries with a
// bounding volume hierarchy).
//
// Binary tree, binned SAH (16 bins per axis on primitive centroids; box
// perimeter in 2D, surface area in 3D), leaves of at most leaf_max primitives.
// Where the remaining depth budget would not fit a balanced subtree the
// split falls back to the centroid median, which bounds the depth by
// kMaxDepth so the traversal's fixed-size stack never overflows.  The tree is
// flattened in depth-first order (a parent precedes its children) with both
// child boxes stored in the parent, so one node fetch (48 B in 2D, 64 B in
// 3D, 16-byte vector loads) decides the visiting order of both children.
//
// Each child also gets a slab: the unit vector n of its elements' summed
// (length- or area-weighted) outward normals and the interval [dmin, dmax]
// of n . v over its vertices, rounded outward.  A point's distance to the
// child's elements is at least max(box distance, distance to the slab), and
// for a patch of a smooth surface the slab is far thinner than the box, so
// closest-point queries near the surface visit fewer nodes.  A child whose
// normals cancel (|sum n| < sum |n| / 2) gets an unbounded slab.  Slabs live
// in a separate array, 2 float4 (2D) or 3 float4 (3D) per node:
//   2D [n0.x n0.y dmin0 dmax0] [n1.x n1.y dmin1 dmax1]
//   3D [n0.x n0.y n0.z dmin0] [dmax0 n1.x n1.y n1.z] [dmin1 dmax1 - -]
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include <vector_types.h>

static inline float4 make_float4(float x, float y, float z, float w) {
  float4 r;
  r.x = x;
  r.y = y;
  r.z = z;
  r.w = w;
  return r;
}

namespace bvc {

// Leaf size (the leaf encoding holds up to 15): measured on GB300 with the
// slab bounds, 2D walks are fastest with ~10 segments per leaf (segment
// tests are cheap, node visits are the divergent part; 14: 1.5% faster,
// 6: 25% slower), 3D walks with 6 triangles (4: 2.5% slower, 8: equal).
#ifndef BVC_LEAF_MAX
#define BVC_LEAF_MAX(dim) ((dim) == 2 ? 10 : 6)
#endif
constexpr int kMaxDepth = 24;  // traversal stacks hold 24 entries
constexpr int kBins = 16;

struct Box {
  float lo[3], hi[3];
  void reset() {
    for (int a = 0; a < 3; ++a) {
      lo[a] = INFINITY;
      hi[a] = -INFINITY;
    }
  }
  void grow(const Box& b) {
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], b.lo[a]);
      hi[a] = std::max(hi[a], b.hi[a]);
    }
  }
  void grow(const float* p) {
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], p[a]);
      hi[a] = std::max(hi[a], p[a]);
    }
  }
  double cost(int dim) const {
    if (lo[0] > hi[0]) return 0.0;
    const double ex = (double)hi[0] - lo[0], ey = (double)hi[1] - lo[1];
    if (dim == 2) return ex + ey;
    const double ez = (double)hi[2] - lo[2];
    return ex * ey + ey * ez + ez * ex;
  }
};

struct Builder {
  int dim;
  int leaf_max;
  std::vector<Box> pbox;
  std::vector<float> cen;  // 3 per prim
  std::vector<int32_t> order;
  std::vector<float4> nodes;
  int per_node;
  std::vector<float4> slabs;
  const float* V = nullptr;
  const int32_t* F = nullptr;

  struct Slab {
    float n[3], dmin, dmax;
  };
  // Slab of the elements order[start .. start + count).
  Slab slab_of(int64_t start, int64_t count) const {
    double S[3] = {0, 0, 0}, A = 0.0;
    for (int64_t i = start; i < start + count; ++i) {
      const int32_t* f = F + (int64_t)order[i] * dim;
      double c[3] = {0, 0, 0};
      if (dim == 2) {
        c[0] = (double)V[2 * f[1] + 1] - V[2 * f[0] + 1];
        c[1] = -((double)V[2 * f[1]] - V[2 * f[0]]);
      } else {
        double e1[3], e2[3];
        for (int a = 0; a < 3; ++a) {
          e1[a] = (double)V[3 * f[1] + a] - V[3 * f[0] + a];
          e2[a] = (double)V[3 * f[2] + a] - V[3 * f[0] + a];
        }
        c[0] = e1[1] * e2[2] - e1[2] * e2[1];
        c[1] = e1[2] * e2[0] - e1[0] * e2[2];
        c[2] = e1[0] * e2[1] - e1[1] * e2[0];
      }
      for (int a = 0; a < 3; ++a) S[a] += c[a];
      A += std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    }
    Slab sl;
    const double L = std::sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
    if (!(L > 0.5 * A) || !(L > 0.0)) {
      sl.n[0] = sl.n[1] = sl.n[2] = 0.0f;
      sl.dmin = -3.0e38f;
      sl.dmax = 3.0e38f;
      return sl;
    }
    for (int a = 0; a < 3; ++a) sl.n[a] = (float)(S[a] / L);
    double lo = INFINITY, hi = -INFINITY;
    for (int64_t i = start; i < start + count; ++i) {
      const int32_t* f = F + (int64_t)order[i] * dim;
      for (int v = 0; v < dim; ++v) {
        double d = 0.0;
        for (int a = 0; a < dim; ++a) d += (double)sl.n[a] * V[(int64_t)f[v] * dim + a];
        lo = std::min(lo, d);
        hi = std::max(hi, d);
      }
    }
    // outward by a relative 2^-20 of the coordinates' scale (the device's
    // FP32 dot product is far more accurate than that)
    double sc = 0.0;
    for (int64_t i = start; i < start + count; ++i) {
      const int32_t* f = F + (int64_t)order[i] * dim;
      for (int v = 0; v < dim; ++v)
        for (int a = 0; a < dim; ++a) sc = std::max(sc, (double)std::fabs(V[(int64_t)f[v] * dim + a]));
    }
    const double pad = std::ldexp(sc, -20);
    sl.dmin = std::nextafter((float)(lo - pad), -INFINITY);
    sl.dmax = std::nextafter((float)(hi + pad), INFINITY);
    return sl;
  }

  void write_slabs(int64_t id, const Slab& L, const Slab& R) {
    float4* q = &slabs[id * (dim == 2 ? 2 : 3)];
    if (dim == 2) {
      q[0] = make_float4(L.n[0], L.n[1], L.dmin, L.dmax);
      q[1] = make_float4(R.n[0], R.n[1], R.dmin, R.dmax);
    } else {
      q[0] = make_float4(L.n[0], L.n[1], L.n[2], L.dmin);
      q[1] = make_float4(L.dmax, R.n[0], R.n[1], R.n[2]);
      q[2] = make_float4(R.dmin, R.dmax, 0.0f, 0.0f);
    }
  }

  static int32_t leaf(int64_t first, int64_t count) { return ~(int32_t)((first << 4) | count); }

  static int ceil_log2(int64_t x) {
    int r = 0;
    while ((int64_t(1) << r) < x) ++r;
    return r;
  }

  int64_t median_split(int64_t start, int64_t count, const Box& cb) {
    int axis = 0;
    for (int a = 1; a < dim; ++a)
      if (cb.hi[a] - cb.lo[a] > cb.hi[axis] - cb.lo[axis]) axis = a;
    const int64_t mid = start + count / 2;
    std::nth_element(order.begin() + start, order.begin() + mid, order.begin() + start + count,
                     [&](int32_t x, int32_t y) {
                       const float a = cen[3 * x + axis], b = cen[3 * y + axis];
                       return a < b || (a == b && x < y);
                     });
    return mid;
  }

  int64_t sah_split(int64_t start, int64_t count, const Box& cb) {
    double best = INFINITY;
    int best_axis = -1, best_bin = -1;
    for (int a = 0; a < dim; ++a) {
      const float ext = cb.hi[a] - cb.lo[a];
      if (!(ext > 0.0f)) continue;
      Box bb[kBins];
      int64_t bn[kBins] = {0};
      for (int b = 0; b < kBins; ++b) bb[b].reset();
      const float sc = kBins / ext;
      for (int64_t i = start; i < start + count; ++i) {
        const int32_t p = order[i];
        int b = (int)((cen[3 * p + a] - cb.lo[a]) * sc);
        b = std::min(std::max(b, 0), kBins - 1);
        bb[b].grow(pbox[p]);
        ++bn[b];
      }
      double lc[kBins];
      int64_t ln[kBins];
      Box acc;
      acc.reset();
      int64_t n = 0;
      for (int b = 0; b < kBins - 1; ++b) {
        acc.grow(bb[b]);
        n += bn[b];
        lc[b] = acc.cost(dim);
        ln[b] = n;
      }
      acc.reset();
      n = 0;
      for (int b = kBins - 1; b > 0; --b) {
        acc.grow(bb[b]);
        n += bn[b];
        if (ln[b - 1] == 0 || n == 0) continue;
        const double c = lc[b - 1] * ln[b - 1] + acc.cost(dim) * n;
        if (c < best) {
          best = c;
          best_axis = a;
          best_bin = b - 1;
        }
      }
    }
    if (best_axis < 0) return -1;
    const float sc = kBins / (cb.hi[best_axis] - cb.lo[best_axis]);
    auto it = std::partition(order.begin() + start, order.begin() + start + count, [&](int32_t p) {
      int b = (int)((cen[3 * p + best_axis] - cb.lo[best_axis]) * sc);
      b = std::min(std::max(b, 0), kBins - 1);
      return b <= best_bin;
    });
    const int64_t mid = it - order.begin();
    if (mid == start || mid == start + count) return -1;
    return mid;
  }

  // Returns the child encoding; fills the subtree's box.
  int32_t build(int64_t start, int64_t count, int depth, Box& out) {
    Box b, cb;
    b.reset();
    cb.reset();
    for (int64_t i = start; i < start + count; ++i) {
      b.grow(pbox[order[i]]);
      cb.grow(&cen[3 * order[i]]);
    }
    out = b;
    if (count <= leaf_max) return leaf(start, count);
    int64_t mid = -1;
    const bool tight = depth + ceil_log2((count + leaf_max - 1) / leaf_max) + 1 >= kMaxDepth;
    if (!tight) mid = sah_split(start, count, cb);
    if (mid < 0) mid = median_split(start, count, cb);
    const int64_t id = (int64_t)nodes.size() / per_node;
    nodes.resize(nodes.size() + per_node);
    slabs.resize(slabs.size() + (dim == 2 ? 2 : 3));
    Box bl, br;
    const int32_t cl = build(start, mid - start, depth + 1, bl);
    const int32_t cr = build(mid, start + count - mid, depth + 1, br);
    write_node(id, bl, br, cl, cr);
    write_slabs(id, slab_of(start, mid - start), slab_of(mid, start + count - mid));
    return (int32_t)id;
  }

  void write_node(int64_t id, const Box& L, const Box& R, int32_t cl, int32_t cr) {
    float4* n = &nodes[id * per_node];
    float ci[2];
    std::memcpy(&ci[0], &cl, 4);
    std::memcpy(&ci[1], &cr, 4);
    if (dim == 2) {
      n[0] = make_float4(L.lo[0], L.lo[1], L.hi[0], L.hi[1]);
      n[1] = make_float4(R.lo[0], R.lo[1], R.hi[0], R.hi[1]);
      n[2] = make_float4(ci[0], ci[1], 0.0f, 0.0f);
    } else {
      n[0] = make_float4(L.lo[0], L.lo[1], L.lo[2], L.hi[0]);
      n[1] = make_float4(L.hi[1], L.hi[2], R.lo[0], R.lo[1]);
      n[2] = make_float4(R.lo[2], R.hi[0], R.hi[1], R.hi[2]);
      n[3] = make_float4(ci[0], ci[1], 0.0f, 0.0f);
    }
  }
};

// Builds the flattened BVH.  prims_out: BVH-ordered primitive records
// (2D: (a, b - a), (1/|b - a|^2, id, 0, 0) with |.|^2 = fma(dy, dy, dx*dx);
// 3D: (a, id), (b - a, 0), (c - a, 0); id stored as int bits), ids_out:
// caller's index per record.  Returns the node count.
int64_t build_bvh(int dim, const float* V, const int32_t* F, int64_t np, std::vector<float4>& nodes_out,
                  std::vector<float4>& prims_out, std::vector<int32_t>& ids_out, std::vector<float4>* slabs_out) {
  Builder B;
  B.dim = dim;
  B.V = V;
  B.F = F;
  B.leaf_max = BVC_LEAF_MAX(dim);
  B.per_node = dim == 2 ? 3 : 4;
  B.pbox.resize(np);
  B.cen.assign(3 * np, 0.0f);
  B.order.resize(np);
  for (int64_t e = 0; e < np; ++e) {
    Box b;
    b.reset();
    double c[3] = {0, 0, 0};
    for (int v = 0; v < dim; ++v) {
      float p[3] = {0, 0, 0};
      for (int a = 0; a < dim; ++a) p[a] = V[(int64_t)F[e * dim + v] * dim + a];
      b.grow(p);
      for (int a = 0; a < dim; ++a) c[a] += p[a];
    }
    for (int a = dim; a < 3; ++a) b.lo[a] = b.hi[a] = 0.0f;
    B.pbox[e] = b;
    for (int a = 0; a < 3; ++a) B.cen[3 * e + a] = (float)(c[a] / dim);
    B.order[e] = (int32_t)e;
  }
  // Root is always an internal node.
  B.nodes.resize(B.per_node);
  B.slabs.resize(dim == 2 ? 2 : 3);
  Box bl, br;
  int32_t cl, cr;
  int64_t mid = np;  // the root's split (np: one leaf child, the other empty)
  if (np <= B.leaf_max) {
    cl = B.build(0, np, 1, bl);
    br.reset();
    cr = Builder::leaf(0, 0);
  } else {
    Box cb;
    cb.reset();
    for (int64_t i = 0; i < np; ++i) cb.grow(&B.cen[3 * i]);
    mid = B.sah_split(0, np, cb);
    if (mid < 0) mid = B.median_split(0, np, cb);
    cl = B.build(0, mid, 1, bl);
    cr = B.build(mid, np - mid, 1, br);
  }
  B.write_node(0, bl, br, cl, cr);
  B.write_slabs(0, B.slab_of(0, mid), B.slab_of(mid, np - mid));
  nodes_out.swap(B.nodes);
  if (slabs_out) slabs_out->swap(B.slabs);
  const int per_prim = dim == 2 ? 2 : 3;
  prims_out.assign(np * per_prim, make_float4(0, 0, 0, 0));
  ids_out.resize(np);
  for (int64_t q = 0; q < np; ++q) {
    const int32_t e = B.order[q];
    ids_out[q] = e;
    const int32_t* f = F + (int64_t)e * dim;
    float idf;
    std::memcpy(&idf, &e, 4);
    if (dim == 2) {
      const float ax = V[2 * f[0]], ay = V[2 * f[0] + 1];
      const float abx = V[2 * f[1]] - ax, aby = V[2 * f[1] + 1] - ay;
      const float den = std::fmaf(aby, aby, abx * abx);
      prims_out[2 * q] = make_float4(ax, ay, abx, aby);
      prims_out[2 * q + 1] = make_float4(1.0f / den, idf, 0.0f, 0.0f);
    } else {
      const float* a = V + 3 * (int64_t)f[0];
      const float* b = V + 3 * (int64_t)f[1];
      const float* c = V + 3 * (int64_t)f[2];
      prims_out[3 * q] = make_float4(a[0], a[1], a[2], idf);
      prims_out[3 * q + 1] = make_float4(b[0] - a[0], b[1] - a[1], b[2] - a[2], 0.0f);
      prims_out[3 * q + 2] = make_float4(c[0] - a[0], c[1] - a[1], c[2] - a[2], 0.0f);
    }
  }
  return (int64_t)nodes_out.size() / B.per_node;
}

}  // namespace bvc
