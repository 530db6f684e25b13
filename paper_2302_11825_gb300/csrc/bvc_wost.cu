// bvc_wost.cu -- mixed Dirichlet / Neumann boundaries: walk on stars
// (Sec. 3.1, Fig. "WoS vs WoSt"), its silhouette and ray queries, the mixed
// cache of Sec. 3.2 (Neumann samples on the boundary with known du/dn,
// Dirichlet samples on the offset boundary) and the pointwise estimator.
//
// Star step at x (Green's second identity on the star region St(x, R) with
// the ball's Green's function G^B, which vanishes on the sphere):
//   a(x) u(x) = int_{dSt} u dG^B/dn + int_St G^B f - int_{dSt_N} G^B h
// with a = 1 inside and 1/2 on a smooth boundary point.  dG^B/dn dz is the
// solid angle over |S|, so a uniform direction (inward hemisphere on the
// boundary, which absorbs the 1/a) and the first crossing of its ray give
// u(next); the source integral in polar form along the same ray, truncated
// at r = min(t_hit, R), and the Neumann term at the crossing (area density
// pdf(w) |n.w| / t^(d-1)) give the per-step weights of bvc.h.
#include <cmath>
#include <cstring>
#include <algorithm>
#include <vector>

#include "bvc_device.cuh"
#include "bvc_internal.h"

namespace bvc {

int64_t build_bvh(int dim, const float* V, const int32_t* F, int64_t np, std::vector<float4>& nodes_out,
                  std::vector<float4>& prims_out, std::vector<int32_t>& ids_out,
                  std::vector<float4>* slabs_out = nullptr);

// Silhouette candidates in BVH order.
//  2D two float4:  (v.x, v.y, n0.x, n0.y) (n1.x, n1.y, always, -)
//  3D four float4: (a.xyz, always) (ab.xyz, 1/|ab|^2) (n0.xyz, -) (n1.xyz, -)
// nodes: the geometry's node layout.
struct DevSil {
  const float4* nodes;
  const float4* prims;
  // per node, per child: a cone (axis.xyz, cos half-angle) holding the normals
  // of every candidate below (cos <= 0: no bound, e.g. an unconditional one)
  const float4* cones;
  int64_t n;        // candidates
  int64_t n_nodes;  // tree nodes
  unsigned long long* stats;  // the whole boundary's status block (debug bounds flag)
  float tau;  // |n_k . a| <= tau counts as zero
  // (1 - gap)^2: a node is visited only when its squared box distance is
  // below shrink2 x the running best (1: the exact closest silhouette)
  float shrink2;
};

// True when no candidate inside the box [lo, hi] under a normal cone can be a
// silhouette seen from x: with psi the angle between the cone axis and the
// direction to the box centre, phi the half-angle the box's bounding sphere
// subtends and theta the cone's half-angle, every n . (p - x) has one sign
// and magnitude above tau when psi + theta + phi < pi/2 (all positive) or
// psi - theta - phi > pi/2 (all negative) (triangle inequality on angles).
// The cone is (axis, cos theta), cos theta <= 0 meaning no bound; the angle
// sums are formed with the addition formulas (no inverse trigonometry).
template <int D>
__device__ __forceinline__ bool cone_prunes(const float4 cone, const float* lo, const float* hi, const float* x,
                                            float tau) {
  if (!(cone.w > 0.0f)) return false;
  float d[3] = {0.0f, 0.0f, 0.0f}, rb2 = 0.0f, dd = 0.0f, ad = 0.0f;
  const float ax[3] = {cone.x, cone.y, cone.z};
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const float h = 0.5f * (hi[a] - lo[a]);
    d[a] = 0.5f * (hi[a] + lo[a]) - x[a];
    rb2 = fmaf(h, h, rb2);
    dd = fmaf(d[a], d[a], dd);
    ad = fmaf(ax[a], d[a], ad);
  }
  if (!(dd > rb2)) return false;
  const float idist = rsqrtf(dd), dist = dd * idist;
  const float sphi = sqrtf(rb2) * idist, cphi = sqrtf(fmaxf(1.0f - sphi * sphi, 0.0f));
  const float cth = cone.w, sth = sqrtf(fmaxf(1.0f - cth * cth, 0.0f));
  // alpha = theta + phi
  const float ca = cth * cphi - sth * sphi, sa = sth * cphi + cth * sphi;
  if (!(ca > 0.0f)) return false;  // theta + phi >= pi/2: the cone spans too much
  const float cpsi = fminf(fmaxf(ad * idist, -1.0f), 1.0f), spsi = sqrtf(fmaxf(1.0f - cpsi * cpsi, 0.0f));
  const float dmin = dist - sqrtf(rb2);
  // psi + alpha < pi/2  <=>  cos psi > sin alpha; margin cos(psi + alpha)
  if (cpsi > sa && (cpsi * ca - spsi * sa) * dmin > tau) return true;
  // psi - alpha > pi/2  <=>  cos psi < -sin alpha; margin -cos(psi - alpha)
  if (cpsi < -sa && -(cpsi * ca + spsi * sa) * dmin > tau) return true;
  return false;
}

}  // namespace bvc

struct bvc_mixed_s {
  int32_t dim;
  bvc_geometry whole, dir, neu;  // owned; neu null without Neumann elements
  int64_t n_dir, n_neu, n_sil, n_sil_nodes;
  double dir_measure, neu_measure;
  void* arena;
  size_t arena_bytes;
  bvc::DevSil sil;
  const int32_t* dir_ids;    // Dirichlet element -> whole element
  const int32_t* neu_local;  // whole element -> Neumann element or -1
  const uint8_t* flags;      // whole element: 1 Neumann
  const double* disp;        // [n_verts][dim] offset displacements from the Dirichlet elements (Sec. 3.2)
  const float2* nmeas;       // Neumann tree: (left, right) subtree measures per node
  const int32_t* neu_q;      // Neumann element -> tree position
};

namespace bvc {

constexpr int kWostBlock = 128;
constexpr int kWStack = kTravStack;
constexpr float kRayInfl = 1e-6f;  // parametric slack of the crossing tests
constexpr int kRecGnW = 0, kRecGradW = 1;

struct WostParams {
  DevGeometry Gd, Gn, Ga;  // Dirichlet part, Neumann part, whole boundary
  DevSil S;
  int32_t has_neu;
  DevFunction g, f, hv, hp;
  const float* starts;  // [D][pt_stride]
  const int32_t* start_elem;
  const float* nrm;
  int64_t pt_stride, i0;
  int32_t W;
  int64_t total;
  uint64_t wid0;
  float eps;
  int32_t max_steps;
  uint64_t seed;
  uint32_t tag;
  float* rec;
  int32_t* steps;
  int32_t* prim;
  const int32_t* neu_local;
  const int32_t* dir_ids;
  const float2* nmeas;  // Neumann tree: subtree measures of each node's children
  const int32_t* neu_q;  // Neumann element -> its position in the Neumann tree's primitive order
  float escape;         // 4 x bounding-box diagonal: a walk farther from the Dirichlet part has escaped
  float sqs;            // sqrt(sigma) of the screened equation (used by the SCR variant)
  unsigned long long* stats;
  unsigned long long* counter;
};

// -------------------------------------------------------------- queries
// Each query is a traversal written as "visit one node" (state: node, stack
// depth sp, the running best) plus a loop over it.  Stacks live in shared
// memory, entry e of a lane at [e * kWostBlock].

// Closest silhouette: one node.  best2 is lowered to the squared distance of
// any nearer silhouette; children are skipped by distance or by their cone.
// With shrink2 < 1 a child whose box is nearer than best2 but not nearer
// than shrink2 x best2 is skipped too, and its squared box distance kept in
// skip2 (the least such): every silhouette point is then at least
// min(best2, skip2) away, a radius no larger than the closest silhouette's.
template <int D>
__device__ __forceinline__ bool sil_visit(const DevSil& S, const float* x, float& best2, float& skip2, int& node,
                                          int& sp, int* snode, float* sdist, TravCount& tcn) {
  ++tcn.nodes;
  if (dbg_bad_at(S.stats, node < 0 || node >= S.n_nodes)) {
    sp = 0;  // abandon the query
    node = -1;
    return true;
  }
  int32_t ch[2];
  float dc[2], blo[2][3], bhi[2][3];
  if (D == 2) {
    const float4 L = __ldg(&S.nodes[3 * node]), R = __ldg(&S.nodes[3 * node + 1]);
    const float4 C = __ldg(&S.nodes[3 * node + 2]);
    dc[0] = box_d2_2(L.x, L.y, L.z, L.w, x);
    dc[1] = box_d2_2(R.x, R.y, R.z, R.w, x);
    ch[0] = __float_as_int(C.x);
    ch[1] = __float_as_int(C.y);
    blo[0][0] = L.x, blo[0][1] = L.y, bhi[0][0] = L.z, bhi[0][1] = L.w;
    blo[1][0] = R.x, blo[1][1] = R.y, bhi[1][0] = R.z, bhi[1][1] = R.w;
  } else {
    const float4 a = __ldg(&S.nodes[4 * node]), b = __ldg(&S.nodes[4 * node + 1]);
    const float4 c = __ldg(&S.nodes[4 * node + 2]), e = __ldg(&S.nodes[4 * node + 3]);
    dc[0] = box_d2_3(a.x, a.y, a.z, a.w, b.x, b.y, x);
    dc[1] = box_d2_3(b.z, b.w, c.x, c.y, c.z, c.w, x);
    ch[0] = __float_as_int(e.x);
    ch[1] = __float_as_int(e.y);
    blo[0][0] = a.x, blo[0][1] = a.y, blo[0][2] = a.z, bhi[0][0] = a.w, bhi[0][1] = b.x, bhi[0][2] = b.y;
    blo[1][0] = b.z, blo[1][1] = b.w, blo[1][2] = c.x, bhi[1][0] = c.y, bhi[1][1] = c.z, bhi[1][2] = c.w;
  }
  bool go[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    go[k] = dc[k] < best2 && !cone_prunes<D>(__ldg(&S.cones[2 * node + k]), blo[k], bhi[k], x, S.tau);
    if (go[k] && !(dc[k] < S.shrink2 * best2)) {
      skip2 = fminf(skip2, dc[k]);
      go[k] = false;
    }
    if (go[k] && ch[k] < 0) {
      const int32_t enc = ~ch[k];
      const int32_t first = enc >> 4, count = enc & 15;
      if (dbg_bad_at(S.stats, first < 0 || (int64_t)first + count > S.n)) {
        go[k] = false;
        continue;
      }
      tcn.prims += (uint32_t)count;
      for (int32_t q = first; q < first + count; ++q) {
        float ax, ay, az = 0.0f, d0, d1, d2;
        bool always;
        if (D == 2) {
          const float4 A = __ldg(&S.prims[2 * q]), B = __ldg(&S.prims[2 * q + 1]);
          ax = A.x - x[0];
          ay = A.y - x[1];
          d0 = fmaf(A.w, ay, A.z * ax);
          d1 = fmaf(B.y, ay, B.x * ax);
          always = B.z != 0.0f;
          d2 = fmaf(ay, ay, ax * ax);
        } else {
          const float4 A = __ldg(&S.prims[4 * q]), B = __ldg(&S.prims[4 * q + 1]);
          const float4 N0 = __ldg(&S.prims[4 * q + 2]), N1 = __ldg(&S.prims[4 * q + 3]);
          ax = A.x - x[0];
          ay = A.y - x[1];
          az = A.z - x[D - 1];
          d0 = fmaf(N0.z, az, fmaf(N0.y, ay, N0.x * ax));
          d1 = fmaf(N1.z, az, fmaf(N1.y, ay, N1.x * ax));
          always = A.w != 0.0f;
          // distance to the edge a + s ab, s in [0, 1]
          const float px = -ax, py = -ay, pz = -az;
          float s = fmaf(B.z, pz, fmaf(B.y, py, B.x * px)) * B.w;
          s = fminf(fmaxf(s, 0.0f), 1.0f);
          const float ex = fmaf(-s, B.x, px), ey = fmaf(-s, B.y, py), ez = fmaf(-s, B.z, pz);
          d2 = fmaf(ez, ez, fmaf(ey, ey, ex * ex));
        }
        const bool z0 = fabsf(d0) <= S.tau, z1 = fabsf(d1) <= S.tau;
        // one element edge-on (zero): a silhouette when the other faces away
        const bool sil = always || (z0 && !z1 && d1 < 0.0f) || (z1 && !z0 && d0 < 0.0f) ||
                         (!z0 && !z1 && ((d0 > 0.0f) != (d1 > 0.0f)));
        if (sil && d2 < best2) best2 = d2;
      }
      go[k] = false;
    }
  }
  // re-test against the bound a leaf may have lowered
#pragma unroll
  for (int k = 0; k < 2; ++k)
    if (go[k] && !(dc[k] < S.shrink2 * best2)) {
      if (dc[k] < best2) skip2 = fminf(skip2, dc[k]);
      go[k] = false;
    }
  if (go[0] && go[1]) {
    const int nearer = dc[1] < dc[0] ? 1 : 0;
    if (!dbg_bad_at(S.stats, sp >= kWStack)) {
      snode[sp * kWostBlock] = ch[1 - nearer];
      sdist[sp * kWostBlock] = dc[1 - nearer];
      ++sp;
    }
    node = ch[nearer];
    return false;
  }
  if (go[0] || go[1]) {
    node = go[0] ? ch[0] : ch[1];
    return false;
  }
  while (sp > 0) {
    --sp;
    const float ds = sdist[sp * kWostBlock];
    if (ds < S.shrink2 * best2) {
      node = snode[sp * kWostBlock];
      return false;
    }
    if (ds < best2) skip2 = fminf(skip2, ds);
  }
  return true;
}

// Closest silhouette point of the Neumann part seen from x, if nearer than
// sqrt(best2): returns min(best2, its squared distance).  With shrink2 < 1 it
// returns a lower bound r2 of that value with r2 >= shrink2 x it: every
// radius up to the star radius keeps the walk's ball star-shaped.
template <int D>
__device__ float sil_closest(const DevSil& S, const float* x, float best2, int* snode, float* sdist, TravCount& tcn) {
  if (S.n == 0) return best2;
  int sp = 0, node = 0;
  float skip2 = __int_as_float(0x7f800000);
  for (int guard = 0; guard < (1 << 22); ++guard)
    if (sil_visit<D>(S, x, best2, skip2, node, sp, snode, sdist, tcn)) break;
  return fminf(best2, skip2);
}

// Entry parameter of the ray o + t w into a box (inv = 1/w with zero
// components replaced by +-1e20), or +inf when it misses within [tmin, tmax].
__device__ __forceinline__ float slab(const float* lo, const float* hi, const float* o, const float* inv, int D,
                                      float tmin, float tmax) {
  float tn = tmin, tf = tmax;
  for (int a = 0; a < D; ++a) {
    const float t0 = (lo[a] - o[a]) * inv[a], t1 = (hi[a] - o[a]) * inv[a];
    tn = fmaxf(tn, fminf(t0, t1));
    tf = fminf(tf, fmaxf(t0, t1));
  }
  // widened exit so that rounding never drops a box the ray grazes
  return tn <= tf * 1.0000004f + 1e-30f ? tn : __int_as_float(0x7f800000);
}

// Visibility rays (vis): elements within kGraze of parallel to the ray are
// not crossings -- a walker on a flat wall looks along it, and a rounded
// near-parallel test there would report a crossing anywhere along the wall.
constexpr float kGraze = 1e-4f;

template <int D>
__device__ __forceinline__ void ray_inv(const float* w, float* inv) {
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const float v = fabsf(w[a]) < 1e-20f ? copysignf(1e-20f, w[a]) : w[a];
    inv[a] = 1.0f / v;
  }
}

// First crossing of o + t w with the Neumann part: one node.  Walk rays (vis
// false) only cross elements they leave the domain through (n . w > 0): a ray
// from inside meets a front face first, and a walker on an edge between two
// Neumann elements must not be stopped by the element it moves away from.
// tmin (<= 0): crossings with t in (tmin, 0] count as crossings at t = 0 --
// that walker, looking out through the other element, must not pass it.
// Elements skip and skip2 are ignored; ties go to the lowest element.
template <int D>
__device__ __forceinline__ bool ray_visit(const DevGeometry& G, const float* o, const float* w, const float* inv,
                                          float tmin, int skip, int skip2, bool vis, float& best, int& bid, int& bq,
                                          int& node, int& sp, int* snode, float* sdist, TravCount& tcn) {
  ++tcn.nodes;
  if (dbg_bad(G, node < 0 || node >= G.n_nodes)) {
    sp = 0;  // abandon the query
    node = -1;
    return true;
  }
  int32_t ch[2];
  float tc[2];
  if (D == 2) {
    const float4 L = __ldg(&G.nodes[3 * node]), R = __ldg(&G.nodes[3 * node + 1]);
    const float4 C = __ldg(&G.nodes[3 * node + 2]);
    const float llo[2] = {L.x, L.y}, lhi[2] = {L.z, L.w}, rlo[2] = {R.x, R.y}, rhi[2] = {R.z, R.w};
    tc[0] = slab(llo, lhi, o, inv, 2, tmin, best);
    tc[1] = slab(rlo, rhi, o, inv, 2, tmin, best);
    ch[0] = __float_as_int(C.x);
    ch[1] = __float_as_int(C.y);
  } else {
    const float4 a = __ldg(&G.nodes[4 * node]), b = __ldg(&G.nodes[4 * node + 1]);
    const float4 c = __ldg(&G.nodes[4 * node + 2]), e = __ldg(&G.nodes[4 * node + 3]);
    const float llo[3] = {a.x, a.y, a.z}, lhi[3] = {a.w, b.x, b.y}, rlo[3] = {b.z, b.w, c.x},
                rhi[3] = {c.y, c.z, c.w};
    tc[0] = slab(llo, lhi, o, inv, 3, tmin, best);
    tc[1] = slab(rlo, rhi, o, inv, 3, tmin, best);
    ch[0] = __float_as_int(e.x);
    ch[1] = __float_as_int(e.y);
  }
  bool go[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    go[k] = tc[k] <= best;
    if (go[k] && ch[k] < 0) {
      const int32_t enc = ~ch[k];
      const int32_t first = enc >> 4, count = enc & 15;
      if (dbg_bad(G, first < 0 || (int64_t)first + count > G.n_prims)) {
        go[k] = false;
        continue;
      }
      tcn.prims += (uint32_t)count;
      for (int32_t q = first; q < first + count; ++q) {
        float tt;
        int id;
        if (D == 2) {
          const float4 Sg = __ldg(&G.prims[2 * q]), T = __ldg(&G.prims[2 * q + 1]);
          id = __float_as_int(T.y);
          const float den = fmaf(w[0], Sg.w, -w[1] * Sg.z);
          if (id == skip || id == skip2 || den == 0.0f) continue;
          if (vis ? fabsf(den) * sqrtf(T.x) < kGraze : !(den > 0.0f)) continue;
          const float qx = Sg.x - o[0], qy = Sg.y - o[1];
          const float s = fmaf(qx, w[1], -qy * w[0]) / den;
          if (!(s >= -kRayInfl && s <= 1.0f + kRayInfl)) continue;
          tt = fmaf(qx, Sg.w, -qy * Sg.z) / den;
        } else {
          // Moller-Trumbore (J. Graphics Tools 2(1), 1997)
          const float4 A = __ldg(&G.prims[3 * q]), B = __ldg(&G.prims[3 * q + 1]), Cc = __ldg(&G.prims[3 * q + 2]);
          id = __float_as_int(A.w);
          if (id == skip || id == skip2) continue;
          const float Px = fmaf(w[1], Cc.z, -w[D - 1] * Cc.y);
          const float Py = fmaf(w[D - 1], Cc.x, -w[0] * Cc.z);
          const float Pz = fmaf(w[0], Cc.y, -w[1] * Cc.x);
          const float det = fmaf(B.z, Pz, fmaf(B.y, Py, B.x * Px));
          if (det == 0.0f) continue;
          if (vis) {
            const float cx = fmaf(B.y, Cc.z, -B.z * Cc.y), cy = fmaf(B.z, Cc.x, -B.x * Cc.z);
            const float cz = fmaf(B.x, Cc.y, -B.y * Cc.x);
            if (fabsf(det) < kGraze * sqrtf(fmaf(cz, cz, fmaf(cy, cy, cx * cx)))) continue;
          } else if (!(det < 0.0f)) {
            continue;  // det = -(n . w) |ab x ac|: a back face
          }
          const float idet = 1.0f / det;
          const float Tx = o[0] - A.x, Ty = o[1] - A.y, Tz = o[D - 1] - A.z;
          const float u = fmaf(Tz, Pz, fmaf(Ty, Py, Tx * Px)) * idet;
          if (!(u >= -kRayInfl && u <= 1.0f + kRayInfl)) continue;
          const float Qx = fmaf(Ty, B.z, -Tz * B.y);
          const float Qy = fmaf(Tz, B.x, -Tx * B.z);
          const float Qz = fmaf(Tx, B.y, -Ty * B.x);
          const float v = fmaf(w[D - 1], Qz, fmaf(w[1], Qy, w[0] * Qx)) * idet;
          if (!(v >= -kRayInfl && u + v <= 1.0f + kRayInfl)) continue;
          tt = fmaf(Cc.z, Qz, fmaf(Cc.y, Qy, Cc.x * Qx)) * idet;
        }
        tt = tt > 0.0f ? tt : (tt > tmin ? 0.0f : -1.0f);
        if (tt >= 0.0f && (tt < best || (tt == best && id < bid))) {
          best = tt;
          bid = id;
          bq = q;
        }
      }
      go[k] = false;
    }
  }
  go[0] = go[0] && tc[0] <= best;
  go[1] = go[1] && tc[1] <= best;
  if (go[0] && go[1]) {
    const int nearer = tc[1] < tc[0] ? 1 : 0;
    if (!dbg_bad(G, sp >= kWStack)) {
      snode[sp * kWostBlock] = ch[1 - nearer];
      sdist[sp * kWostBlock] = tc[1 - nearer];
      ++sp;
    }
    node = ch[nearer];
    return false;
  }
  if (go[0] || go[1]) {
    node = go[0] ? ch[0] : ch[1];
    return false;
  }
  while (sp > 0) {
    --sp;
    if (sdist[sp * kWostBlock] <= best) {
      node = snode[sp * kWostBlock];
      return false;
    }
  }
  return true;
}

// Outward unit normal of the Neumann element at tree position q.
template <int D>
__device__ __forceinline__ void neumann_normal(const DevGeometry& G, int q, float* n) {
  if (D == 2) {
    const float4 Sg = __ldg(&G.prims[2 * q]), T = __ldg(&G.prims[2 * q + 1]);
    const float il = sqrtf(T.x);
    n[0] = Sg.w * il;
    n[D - 1] = -Sg.z * il;
  } else {
    const float4 B = __ldg(&G.prims[3 * q + 1]), Cc = __ldg(&G.prims[3 * q + 2]);
    const float cx = fmaf(B.y, Cc.z, -B.z * Cc.y), cy = fmaf(B.z, Cc.x, -B.x * Cc.z), cz = fmaf(B.x, Cc.y, -B.y * Cc.x);
    const float il = rsqrtf(fmaf(cz, cz, fmaf(cy, cy, cx * cx)));
    n[0] = cx * il;
    n[1] = cy * il;
    n[D - 1] = cz * il;
  }
}

// First crossing of o + t w, 0 < t <= tmax (see ray_visit): the element's
// Neumann id or -1; t and its outward normal through t_out, n.
template <int D, bool VIS = false>
__device__ int ray_first(const DevGeometry& G, const float* o, const float* w, float tmax, int skip, int skip2,
                         float tmin, float& t_out, float* n, int* snode, float* sdist, TravCount& tcn) {
  float inv[D];
  ray_inv<D>(w, inv);
  float best = tmax;
  int bid = 0x7fffffff, bq = -1;
  int sp = 0, node = 0;
  for (int guard = 0; guard < (1 << 22); ++guard)
    if (ray_visit<D>(G, o, w, inv, tmin, skip, skip2, VIS, best, bid, bq, node, sp, snode, sdist, tcn)) break;
  if (bq < 0) {
    t_out = __int_as_float(0x7f800000);
    return -1;
  }
  t_out = best;
  neumann_normal<D>(G, bq, n);
  return bid;
}

// A uniform per level of the area-sampling descent: an integer hash of the
// draw's words x, y and the level (xor-shift-multiply rounds, constants of
// C. Wellons' "lowbias32").
__device__ __forceinline__ float level_uniform(const U4& r, uint32_t lv) {
  uint32_t v = r.x ^ (r.y + 0x9e3779b9u * (lv + 1u));
  v ^= v >> 16;
  v *= 0x7feb352du;
  v ^= v >> 15;
  v *= 0x846ca68bu;
  v ^= v >> 16;
  return u01f(v);
}

// A point z on the Neumann part, chosen by descending the Neumann tree:
// at each node a child whose box reaches into B(x, R) is taken with
// probability proportional to its subtree measure (nm[node] = (left, right)),
// in the leaf an element by its measure, on the element a uniform point
// (2D a + s ab; 3D barycentrics (1 - sqrt u1, sqrt u1 (1 - u2), sqrt u1 u2)).
// Every Neumann point inside the ball has positive density; ipdf = 1/pdf(z).
// Draw words: x, y seed one uniform per level (and the leaf's element
// choice), z, w place the point.  One level per call: returns 0 to go on,
// 1 with the point, 2 when no subtree reaches into the ball.
template <int D>
__device__ __forceinline__ int descent_visit(const DevGeometry& G, const float2* __restrict__ nm, const float* x,
                                             float R2, const U4& r, int& level, int& node, float& pdf, float* z,
                                             float* nz, int& id, float& ipdf, TravCount& tcn) {
  ++tcn.nodes;
  if (dbg_bad(G, node < 0 || node >= G.n_nodes)) return 2;
  int32_t ch[2];
  float dc[2];
  if (D == 2) {
    const float4 L = __ldg(&G.nodes[3 * node]), Rb = __ldg(&G.nodes[3 * node + 1]);
    const float4 C = __ldg(&G.nodes[3 * node + 2]);
    dc[0] = box_d2_2(L.x, L.y, L.z, L.w, x);
    dc[1] = box_d2_2(Rb.x, Rb.y, Rb.z, Rb.w, x);
    ch[0] = __float_as_int(C.x);
    ch[1] = __float_as_int(C.y);
  } else {
    const float4 a = __ldg(&G.nodes[4 * node]), b = __ldg(&G.nodes[4 * node + 1]);
    const float4 c = __ldg(&G.nodes[4 * node + 2]), e = __ldg(&G.nodes[4 * node + 3]);
    dc[0] = box_d2_3(a.x, a.y, a.z, a.w, b.x, b.y, x);
    dc[1] = box_d2_3(b.z, b.w, c.x, c.y, c.z, c.w, x);
    ch[0] = __float_as_int(e.x);
    ch[1] = __float_as_int(e.y);
  }
  const float2 m = __ldg(&nm[node]);
  const float w0 = dc[0] < R2 ? m.x : 0.0f, w1 = dc[1] < R2 ? m.y : 0.0f;
  if (!(w0 + w1 > 0.0f) || level >= 63) return 2;
  const float p0 = w0 / (w0 + w1);
  const int pick = level_uniform(r, (uint32_t)level) < p0 ? 0 : 1;
  pdf *= pick == 0 ? p0 : 1.0f - p0;
  ++level;
  if (ch[pick] >= 0) {
    node = ch[pick];
    return 0;
  }
  // leaf: an element by measure
  const int32_t enc = ~ch[pick];
  const int32_t first = enc >> 4, count = enc & 15;
  auto elem_measure = [&](int32_t q) {
    if (D == 2) return 1.0f / sqrtf(__ldg(&G.prims[2 * q + 1]).x);
    const float4 B = __ldg(&G.prims[3 * q + 1]), Cc = __ldg(&G.prims[3 * q + 2]);
    const float cx = fmaf(B.y, Cc.z, -B.z * Cc.y), cy = fmaf(B.z, Cc.x, -B.x * Cc.z);
    const float cz = fmaf(B.x, Cc.y, -B.y * Cc.x);
    return 0.5f * sqrtf(fmaf(cz, cz, fmaf(cy, cy, cx * cx)));
  };
  if (dbg_bad(G, first < 0 || count == 0 || (int64_t)first + count > G.n_prims)) return 2;
  tcn.prims += (uint32_t)count;
  float tot = 0.0f;
  for (int32_t q = first; q < first + count; ++q) tot += elem_measure(q);
  if (!(tot > 0.0f)) return 2;
  const float target = level_uniform(r, 63u) * tot;
  float run = 0.0f;
  int32_t qs = first + count - 1;
  for (int32_t q = first; q < first + count; ++q) {
    run += elem_measure(q);
    if (run > target) {
      qs = q;
      break;
    }
  }
  // pdf(z) = (descent probability) x (m_e / tot) x (1 / m_e)
  ipdf = tot / pdf;
  const float s1 = u01f(r.z), s2 = u01f(r.w);
  if (D == 2) {
    const float4 S = __ldg(&G.prims[2 * qs]), T = __ldg(&G.prims[2 * qs + 1]);
    z[0] = fmaf(s1, S.z, S.x);
    z[D - 1] = fmaf(s1, S.w, S.y);
    id = __float_as_int(T.y);
  } else {
    const float4 A = __ldg(&G.prims[3 * qs]), B = __ldg(&G.prims[3 * qs + 1]), Cc = __ldg(&G.prims[3 * qs + 2]);
    const float sq = sqrtf(s1), b1 = sq * (1.0f - s2), b2 = sq * s2;
    z[0] = fmaf(b2, Cc.x, fmaf(b1, B.x, A.x));
    z[1] = fmaf(b2, Cc.y, fmaf(b1, B.y, A.y));
    z[D - 1] = fmaf(b2, Cc.z, fmaf(b1, B.z, A.z));
    id = __float_as_int(A.w);
  }
  neumann_normal<D>(G, qs, nz);
  return 1;
}

template <int D>
__device__ bool sample_neumann(const DevGeometry& G, const float2* __restrict__ nm, const float* x, float R,
                               const U4 r, float* z, float* nz, int& id, float& ipdf, TravCount& tcn) {
  float pdf = 1.0f;
  int node = 0, level = 0;
  for (;;) {
    const int st = descent_visit<D>(G, nm, x, R * R, r, level, node, pdf, z, nz, id, ipdf, tcn);
    if (st) return st == 1;
  }
}

// The Neumann term over the element under an on-boundary x (Neumann id
// self at tree position q), sampled around x inside the element, where G^B
// is singular: 2D a side (u0 < 1/2: towards b) and rho = u1 rho_max with
// rho_max = min(R, distance to that end); 3D a direction theta = 2 pi u0 in
// the element's plane (e1 = ab / |ab|, e2 = n x e1) and rho = u1 rho_max,
// rho_max = min(R, distance to the triangle's border along it).  Returns the
// point, the element normal and 1/pdf (2 rho_max in 2D, 2 pi rho rho_max in
// 3D), or false when x is not inside the element.
template <int D>
__device__ bool sample_own(const DevGeometry& G, int q, const float* x, float R, float u0, float u1, float* z,
                           float* nz, float& rho, float& ipdf) {
  if (D == 2) {
    const float4 S = __ldg(&G.prims[2 * q]), T = __ldg(&G.prims[2 * q + 1]);
    const float il = sqrtf(T.x), len = 1.0f / il;
    const float tx = S.z * il, ty = S.w * il;
    float sx = fmaf(x[D - 1] - S.y, ty, (x[0] - S.x) * tx);
    sx = fminf(fmaxf(sx, 0.0f), len);
    const float sg = u0 < 0.5f ? 1.0f : -1.0f;
    const float rmax = fminf(R, sg > 0.0f ? len - sx : sx);
    if (!(rmax > 0.0f)) return false;
    rho = u1 * rmax;
    z[0] = fmaf(sg * rho, tx, x[0]);
    z[D - 1] = fmaf(sg * rho, ty, x[D - 1]);
    nz[0] = ty;
    nz[D - 1] = -tx;
    ipdf = 2.0f * rmax;
    return true;
  } else {
    const float4 A = __ldg(&G.prims[3 * q]), B = __ldg(&G.prims[3 * q + 1]), Cc = __ldg(&G.prims[3 * q + 2]);
    float n[3] = {fmaf(B.y, Cc.z, -B.z * Cc.y), fmaf(B.z, Cc.x, -B.x * Cc.z), fmaf(B.x, Cc.y, -B.y * Cc.x)};
    const float inn = rsqrtf(fmaf(n[2], n[2], fmaf(n[1], n[1], n[0] * n[0])));
    const float il1 = rsqrtf(fmaf(B.z, B.z, fmaf(B.y, B.y, B.x * B.x)));
    float e1[3] = {B.x * il1, B.y * il1, B.z * il1};
#pragma unroll
    for (int k = 0; k < 3; ++k) n[k] *= inn;
    const float e2[3] = {n[1] * e1[2] - n[2] * e1[1], n[2] * e1[0] - n[0] * e1[2], n[0] * e1[1] - n[1] * e1[0]};
    float sn, cs;
    sincospif(2.0f * u0, &sn, &cs);
    float d[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) d[k] = fmaf(cs, e1[k], sn * e2[k]);
    // vertices relative to x, and the in-plane inward normals of the edges
    const float P[3][3] = {{A.x - x[0], A.y - x[1], A.z - x[D - 1]},
                           {A.x + B.x - x[0], A.y + B.y - x[1], A.z + B.z - x[D - 1]},
                           {A.x + Cc.x - x[0], A.y + Cc.y - x[1], A.z + Cc.z - x[D - 1]}};
    float rmax = R;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int jn = j == 2 ? 0 : j + 1;
      const float pq[3] = {P[jn][0] - P[j][0], P[jn][1] - P[j][1], P[jn][2] - P[j][2]};
      const float m[3] = {n[1] * pq[2] - n[2] * pq[1], n[2] * pq[0] - n[0] * pq[2], n[0] * pq[1] - n[1] * pq[0]};
      const float dm = fmaf(d[2], m[2], fmaf(d[1], m[1], d[0] * m[0]));
      if (dm < 0.0f) {
        // (x - p) . m over -(d . m), with x - p = -P[j]
        const float lim = -fmaf(P[j][2], m[2], fmaf(P[j][1], m[1], P[j][0] * m[0])) / -dm;
        rmax = fminf(rmax, lim);
      }
    }
    if (!(rmax > 0.0f)) return false;
    rho = u1 * rmax;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      z[k < D ? k : 0] = fmaf(rho, d[k], x[k < D ? k : 0]);
      nz[k < D ? k : 0] = n[k];
    }
    ipdf = 2.0f * kPiF * rho * rmax;
    return true;
  }
}

template <int D>
__device__ __forceinline__ float neumann_h(const DevFunction& hv, const DevFunction& hp, const float* z,
                                           const float* n) {
  float v = hv.n_terms > 0 ? eval_fn<D>(hv, z) : 0.0f;
  if (hp.n_terms > 0) {
    float gr[D];
    eval_fn_grad<D>(hp, z, gr);
#pragma unroll
    for (int a = 0; a < D; ++a) v = fmaf(n[a], gr[a], v);
  }
  return v;
}

template <int D>
__global__ void __launch_bounds__(128) k_mixed_query(DevGeometry Gd, DevSil S, const float* __restrict__ pts,
                                                     int64_t m, float* __restrict__ d_dir,
                                                     float* __restrict__ d_sil) {
  __shared__ int snode[kWStack * kWostBlock];
  __shared__ float sdist[kWStack * kWostBlock];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    float p[D];
#pragma unroll
    for (int a = 0; a < D; ++a) p[a] = pts[a * m + i];
    Hit<D> h;
    TravCount tc{0, 0};
    bvh_closest<D>(Gd, p, h, snode + threadIdx.x, sdist + threadIdx.x, kWostBlock, tc);
    if (d_dir) d_dir[i] = sqrtf(h.d2);
    if (d_sil) d_sil[i] = sqrtf(sil_closest<D>(S, p, __int_as_float(0x7f800000), snode + threadIdx.x,
                                               sdist + threadIdx.x, tc));
  }
}

template <int D>
__global__ void __launch_bounds__(128) k_mixed_rays(DevGeometry Gn, int32_t has_neu, const float* __restrict__ org,
                                                    const float* __restrict__ dir, const int32_t* __restrict__ skip,
                                                    int64_t m, float tmax, float* __restrict__ t_out,
                                                    int32_t* __restrict__ e_out) {
  __shared__ int snode[kWStack * kWostBlock];
  __shared__ float sdist[kWStack * kWostBlock];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    float o[D], w[D], n[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      o[a] = org[a * m + i];
      w[a] = dir[a * m + i];
    }
    float t = __int_as_float(0x7f800000);
    int e = -1;
    if (has_neu) {
      TravCount tc{0, 0};
      e = ray_first<D>(Gn, o, w, tmax, skip ? skip[i] : -1, -1, -Gn.tau, t, n, snode + threadIdx.x,
                       sdist + threadIdx.x, tc);
    }
    t_out[i] = t;
    e_out[i] = e;
  }
}

// ------------------------------------------------------------ the walk
// One walk per lane, advanced one step per loop iteration; a lane whose walk
// ends takes the next walk at once (the warp's idle lanes share one atomic
// on the work counter), so long walks do not idle the rest of the warp.
// Resident blocks per SM the walk-on-stars kernel is compiled for (measured
// best on GB300 for the 20k-segment mixed star: 4).
#ifndef BVC_WOST_MINB
#define BVC_WOST_MINB 4
#endif
// SCR: the screened equation (Delta - sigma) u = f: the gradient ball
// multiplies the walk's throughput by its mean-value factor C and scales
// the gradient by Qg (screened_factors); a star step whose direction meets
// the boundary at distance r multiplies it by W(r) (star_kernel_sigma); the
// step's source and Neumann terms use the ball's screened Green's function
// (screened_step_weights, ball_green_sigma) and the throughput into the step.
template <int D, bool HAS_F, bool HAS_H, int REC, bool SCR>
__global__ void __launch_bounds__(kWostBlock, BVC_WOST_MINB) k_wost(const WostParams P) {
  __shared__ int snode[kWStack * kWostBlock];
  __shared__ float sdist[kWStack * kWostBlock];
  int* const sn = snode + threadIdx.x;
  float* const sd = sdist + threadIdx.x;
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  unsigned long long my_steps = 0, my_capped = 0;
  TravCount tc{0, 0};  // node fetches and primitive tests of every query
  bool active = false, more = true;
  // walk state
  int64_t t = 0, i = 0;
  float x[D], nx[D], nu[D], pbar[D];
#pragma unroll
  for (int a = 0; a < D; ++a) x[a] = nx[a] = nu[a] = pbar[a] = 0.0f;
  bool on_n = false, start_on_n = false;
  int self = -1, k = 0;
  float acc = 0.0f, wf0 = 0.0f, wg0 = 0.0f, R0 = 0.0f, cv = 0.0f;
  float thr = 1.0f, C0 = 1.0f, Qg0 = 1.0f;  // screened: throughput, gradient ball's factors
  Hit<D> h;
  for (;;) {
    // ---- idle lanes take the next walks
    const unsigned need = __ballot_sync(FULL, !active);
    if (need != 0u && more) {
      const unsigned nneed = (unsigned)__popc(need);
      unsigned long long base = 0;
      if (lane == 0) base = atomicAdd(P.counter, (unsigned long long)nneed);
      base = __shfl_sync(FULL, base, 0);
      if ((int64_t)(base + nneed) >= P.total) more = false;
      if (!active) {
        const int64_t tt = (int64_t)base + __popc(need & ((1u << lane) - 1u));
        if (tt < P.total) {
          active = true;
          t = tt;
          i = P.i0 + t / P.W;
#pragma unroll
          for (int a = 0; a < D; ++a) {
            x[a] = P.starts[a * P.pt_stride + i];
            nx[a] = nu[a] = 0.0f;
          }
          on_n = false;
          self = -1;
          if (P.start_elem != nullptr && P.has_neu) {
            const int32_t e0 = P.start_elem[i];
            if (e0 >= 0 && e0 < P.Ga.n_prims) {
              const int32_t nl = P.neu_local[e0];
              if (nl >= 0) {
                on_n = true;
                self = nl;
#pragma unroll
                for (int a = 0; a < D; ++a) nx[a] = P.nrm[a * P.pt_stride + i];
              }
            }
          }
          start_on_n = on_n;
          acc = wf0 = wg0 = R0 = cv = 0.0f;
          if (SCR) thr = C0 = Qg0 = 1.0f;
          k = 0;
        }
      }
    }
    if (__ballot_sync(FULL, active) == 0u) break;
    if (!active) continue;
    // ---- one step of this lane's walk
    bvh_closest<D, true>(P.Gd, x, h, sn, sd, kWostBlock, tc);
#pragma unroll
    for (int a = 0; a < D; ++a) pbar[a] = x[a] - h.df[a];
    const float dD = sqrtf(h.d2);
    ++k;
    bool done = false, reached = false;
    if (!(dD <= P.escape)) {
      done = true;  // left the domain through a rounding gap: capped
    } else {
      if (k == 1) cv = eval_fn<D, true>(P.g, pbar);  // control variate of the gradient
      if (dD < P.eps) {
        done = reached = true;
      } else if (k >= P.max_steps) {
        done = true;
      }
    }
    if (!done) {
      const U4 rr = philox_draw(P.seed, P.wid0 + (uint64_t)t, (uint32_t)(k - 1), P.tag);
      const float u0 = u01f(rr.x), u2 = u01f(rr.z);
      float om[D];
      if (D == 2) {
        float sn2, cs;
        sincospif(2.0f * u0, &sn2, &cs);
        om[0] = cs;
        om[D - 1] = sn2;
      } else {
        const float u1 = u01f(rr.y);
        const float zc = 1.0f - 2.0f * u0;
        const float st = 2.0f * sqrtf(u0 * (1.0f - u0));
        float sn2, cs;
        sincospif(2.0f * u1, &sn2, &cs);
        om[0] = st * cs;
        om[1] = st * sn2;
        om[D - 1] = zc;
      }
      bool ball = false;
      if (k == 1 && !on_n) {
        Hit<D> ha;
        bvh_closest<D, true>(P.Ga, x, ha, sn, sd, kWostBlock, tc);
        const float dA = sqrtf(ha.d2);
        if (dA >= P.eps) {
          // the gradient ball B(x, d_all): no boundary inside
          ball = true;
          const float R = dA;
          if (SCR) {
            screened_factors<D>(P.sqs * R, C0, Qg0);
            thr = C0;
          }
          if (HAS_F) {
            const float rho = R * u2;
            float y[D];
#pragma unroll
            for (int a = 0; a < D; ++a) y[a] = fmaf(rho, om[a], x[a]);
            const float fy = eval_fn<D, true>(P.f, y);
            float wu = D == 2 ? R * rho * __logf(u2) : -rho * (R - rho), wg = 0.0f;
            if (SCR) screened_step_weights<D>(P.sqs, R, rho, true, wu, wg);
            acc = fmaf(wu, fy, acc);
            wf0 = wu * fy;
            const float q = D == 2 ? u2 * u2 : u2 * u2 * u2;
            wg0 = (SCR ? wg : -R * (1.0f - q)) * fy;
          }
          R0 = R;
#pragma unroll
          for (int a = 0; a < D; ++a) {
            nu[a] = om[a];
            x[a] = fmaf(R, om[a], x[a]);
          }
        }
      }
      if (!ball) {
        // star step
        if (on_n) {
          float sdot = 0.0f;
#pragma unroll
          for (int a = 0; a < D; ++a) sdot = fmaf(nx[a], om[a], sdot);
          if (sdot > 0.0f)
#pragma unroll
            for (int a = 0; a < D; ++a) om[a] = -om[a];
        }
        float R = dD;
        int eh = -1;
        float th = 0.0f, nh[D];
        if (P.has_neu) {
          R = sqrtf(sil_closest<D>(P.S, x, h.d2, sn, sd, tc));
          R = fmaxf(R, P.eps);
          eh = ray_first<D>(P.Gn, x, om, R, on_n ? self : -1, -1, -P.Gn.tau, th, nh, sn, sd, tc);
        }
        const float rl = eh >= 0 ? th : R;
        if (HAS_F && rl > 0.0f) {  // a crossing at t = 0 leaves no segment
          const float rho = rl * u2;
          float y[D];
#pragma unroll
          for (int a = 0; a < D; ++a) y[a] = fmaf(rho, om[a], x[a]);
          float wu = D == 2 ? rl * rho * __logf(rho / R) : -rl * rho * (1.0f - rho / R);
          if (SCR) {
            // the ball's weight at rho, scaled by r / R (rho is uniform on [0, r])
            float wb, wgb;
            screened_step_weights<D>(P.sqs, R, rho, false, wb, wgb);
            wu = thr * (rl / R) * wb;
          }
          acc = fmaf(wu, eval_fn<D, true>(P.f, y), acc);
        }
        if (HAS_H && P.has_neu) {
          // area-sampled Neumann term over the part inside B(x, R)
          const U4 r2 = philox_draw(P.seed, P.wid0 + (uint64_t)t, (uint32_t)(k - 1), P.tag + 8u);
          float z[D], nz[D], ipdf;
          int ez;
          // the element under an on-boundary x: sampled around x below
          if (sample_neumann<D>(P.Gn, P.nmeas, x, R, r2, z, nz, ez, ipdf, tc) && !(on_n && ez == self)) {
            float dz[D], r2z = 0.0f;
#pragma unroll
            for (int a = 0; a < D; ++a) {
              dz[a] = z[a] - x[a];
              r2z = fmaf(dz[a], dz[a], r2z);
            }
            const float rz = sqrtf(r2z);
            if (rz < R && rz > 0.0f) {
              const float ir = 1.0f / rz;
#pragma unroll
              for (int a = 0; a < D; ++a) dz[a] *= ir;
              float tv, nv[D];
              const int ev =
                  ray_first<D, true>(P.Gn, x, dz, rz * (1.0f - 1e-5f), on_n ? self : -1, ez, 0.0f, tv, nv, sn, sd, tc);
              if (ev < 0) {
                // G^B of -Laplacian: ln(R/r)/(2 pi) (2D), (1/r - 1/R)/(4 pi) (3D)
                const float gb = SCR ? thr * ball_green_sigma<D>(P.sqs, R, rz)
                                     : (D == 2 ? __logf(R * ir) * (0.5f / kPiF) : (ir - 1.0f / R) * (0.25f / kPiF));
                acc = fmaf((on_n ? 2.0f : 1.0f) * gb * ipdf, neumann_h<D>(P.hv, P.hp, z, nz), acc);
              }
            }
          }
          if (on_n) {
            const U4 r3 = philox_draw(P.seed, P.wid0 + (uint64_t)t, (uint32_t)(k - 1), P.tag + 12u);
            float rho;
            if (sample_own<D>(P.Gn, P.neu_q[self], x, R, u01f(r3.x), u01f(r3.y), z, nz, rho, ipdf)) {
              const float gb = SCR ? thr * ball_green_sigma<D>(P.sqs, R, rho)
                                   : (D == 2 ? __logf(R / rho) * (0.5f / kPiF)
                                             : (1.0f / rho - 1.0f / R) * (0.25f / kPiF));
              acc = fmaf(2.0f * gb * ipdf, neumann_h<D>(P.hv, P.hp, z, nz), acc);
            }
          }
        }
        if (SCR) thr *= star_kernel_sigma<D>(P.sqs, R, rl);
        if (eh >= 0) {
#pragma unroll
          for (int a = 0; a < D; ++a) {
            x[a] = fmaf(th, om[a], x[a]);
            nx[a] = nh[a];
          }
          on_n = true;
          self = eh;
        } else {
#pragma unroll
          for (int a = 0; a < D; ++a) x[a] = fmaf(R, om[a], x[a]);
          on_n = false;
          self = -1;
        }
      }
      continue;
    }
    // ---- the walk ended: its records
    const float gend = eval_fn<D, true>(P.g, pbar);
    const float U = (SCR ? thr * gend : gend) + acc;
    // screened: (U - wf0) / C0 estimates u at the gradient ball's sphere point
    const float sc = !(R0 > 0.0f) ? 0.0f
                     : SCR       ? fmaf(((float)D / R0) * Qg0, (U - wf0) / C0 - cv, wg0)
                                 : ((float)D / R0) * (U - wf0 - cv) + wg0;
    P.rec[t] = U;
    if (REC == kRecGnW) {
      float v;
      if (start_on_n) {
        float z0[D], n0[D];
#pragma unroll
        for (int a = 0; a < D; ++a) {
          z0[a] = P.starts[a * P.pt_stride + i];
          n0[a] = P.nrm[a * P.pt_stride + i];
        }
        v = neumann_h<D>(P.hv, P.hp, z0, n0);
      } else {
        float nn2 = 0.0f;
#pragma unroll
        for (int a = 0; a < D; ++a) nn2 = fmaf(P.nrm[a * P.pt_stride + i], nu[a], nn2);
        v = sc * nn2;
      }
      P.rec[P.total + t] = v;
    } else {
#pragma unroll
      for (int a = 0; a < D; ++a) P.rec[(1 + a) * P.total + t] = sc * nu[a];
    }
    if (P.steps) P.steps[t] = k;
    if (P.prim) P.prim[t] = h.id >= 0 && h.id < 0x7fffffff ? P.dir_ids[h.id] : -1;
    my_steps += (unsigned long long)k;
    if (!reached) ++my_capped;
    active = false;
  }
  unsigned long long my_nodes = tc.nodes, my_prims = tc.prims;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    my_steps += __shfl_xor_sync(FULL, my_steps, o);
    my_capped += __shfl_xor_sync(FULL, my_capped, o);
    my_nodes += __shfl_xor_sync(FULL, my_nodes, o);
    my_prims += __shfl_xor_sync(FULL, my_prims, o);
  }
  if (lane == 0) {
    if (my_steps) atomicAdd(&P.stats[kStatSteps], my_steps);
    if (my_capped) atomicAdd(&P.stats[kStatCapped], my_capped);
    if (my_nodes) atomicAdd(&P.stats[kStatNodes], my_nodes);
    if (my_prims) atomicAdd(&P.stats[kStatPrims], my_prims);
  }
}

// The screened variant always runs the Neumann term (zero data adds zeros).
template <int D, int REC>
static const void* wost_kernel(bool has_f, bool has_h, bool scr) {
  if (scr) return has_f ? (const void*)k_wost<D, true, true, REC, true> : (const void*)k_wost<D, false, true, REC, true>;
  if (has_f)
    return has_h ? (const void*)k_wost<D, true, true, REC, false> : (const void*)k_wost<D, true, false, REC, false>;
  return has_h ? (const void*)k_wost<D, false, true, REC, false> : (const void*)k_wost<D, false, false, REC, false>;
}

static bvc_status launch_wost(int dim, int rec, const WostParams& P, cudaStream_t s) {
  const bool hf = P.f.n_terms > 0, hh = P.hv.n_terms > 0 || P.hp.n_terms > 0, sc = P.sqs > 0.0f;
  const void* kern = dim == 2 ? (rec == kRecGnW ? wost_kernel<2, kRecGnW>(hf, hh, sc)
                                                : wost_kernel<2, kRecGradW>(hf, hh, sc))
                              : (rec == kRecGnW ? wost_kernel<3, kRecGnW>(hf, hh, sc)
                                                : wost_kernel<3, kRecGradW>(hf, hh, sc));
  const int bps = max_blocks_per_sm(kern, kWostBlock, 0);
  int64_t grid = (int64_t)num_sms() * (bps > 0 ? bps : 1);
  const int64_t need = (P.total + kWostBlock - 1) / kWostBlock;
  if (need < grid) grid = need > 0 ? need : 1;
  BVC_CUDA_TRY(cudaMemsetAsync(P.counter, 0, sizeof(unsigned long long), s));
  WostParams Q = P;
  void* args[] = {(void*)&Q};
  ProfScope ps("wost_walk", s);
  BVC_CUDA_TRY(cudaLaunchKernel(kern, dim3((unsigned)grid), dim3(kWostBlock), args, 0, s));
  return BVC_OK;
}

__global__ void k_mixed_add_count(int64_t* counts, int64_t w) {
  if (threadIdx.x == 0 && blockIdx.x == 0) counts[0] += w;
}

// ------------------------------------------------------------ host side
static double elem_normal(int dim, const float* V, const int32_t* f, double* n) {
  if (dim == 2) {
    const double dx = (double)V[2 * f[1]] - V[2 * f[0]], dy = (double)V[2 * f[1] + 1] - V[2 * f[0] + 1];
    const double len = std::sqrt(dx * dx + dy * dy);
    n[0] = dy / len;
    n[1] = -dx / len;
    return len;
  }
  double e1[3], e2[3];
  for (int a = 0; a < 3; ++a) {
    e1[a] = (double)V[3 * f[1] + a] - V[3 * f[0] + a];
    e2[a] = (double)V[3 * f[2] + a] - V[3 * f[0] + a];
  }
  const double c[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
  const double len = std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
  for (int a = 0; a < 3; ++a) n[a] = c[a] / len;
  return 0.5 * len;
}

struct SilCand {
  int32_t a, b;       // vertex (2D: a == b) or edge
  int32_t e0, e1;     // the two Neumann elements, or -1
  bool always;
};

// Silhouette candidates: vertices (2D) / edges (3D) whose elements are all
// Neumann; two elements give a candidate with both normals, one or more
// than two an unconditional one.
static std::vector<SilCand> silhouette_candidates(int dim, int64_t n_verts, const int32_t* F, int64_t np,
                                                  const uint8_t* neu) {
  std::vector<SilCand> out;
  if (dim == 2) {
    std::vector<int32_t> nn(n_verts, 0), nd(n_verts, 0), first(n_verts, -1), second(n_verts, -1);
    for (int64_t e = 0; e < np; ++e)
      for (int k = 0; k < 2; ++k) {
        const int32_t v = F[2 * e + k];
        if (!neu[e]) {
          ++nd[v];
        } else {
          if (nn[v] == 0) first[v] = (int32_t)e;
          else if (nn[v] == 1) second[v] = (int32_t)e;
          ++nn[v];
        }
      }
    for (int64_t v = 0; v < n_verts; ++v) {
      if (nn[v] == 0 || nd[v] > 0) continue;
      out.push_back({(int32_t)v, (int32_t)v, first[v], second[v], nn[v] != 2});
    }
    return out;
  }
  struct ER {
    int32_t lo, hi, e;
  };
  std::vector<ER> ed;
  ed.reserve((size_t)np * 3);
  for (int64_t e = 0; e < np; ++e)
    for (int k = 0; k < 3; ++k) {
      const int32_t a = F[3 * e + k], b = F[3 * e + (k + 1) % 3];
      ed.push_back({std::min(a, b), std::max(a, b), (int32_t)e});
    }
  std::sort(ed.begin(), ed.end(), [](const ER& x, const ER& y) {
    return x.lo != y.lo ? x.lo < y.lo : (x.hi != y.hi ? x.hi < y.hi : x.e < y.e);
  });
  for (size_t i = 0; i < ed.size();) {
    size_t j = i;
    int n_n = 0, n_d = 0;
    int32_t en[2] = {-1, -1};
    for (; j < ed.size() && ed[j].lo == ed[i].lo && ed[j].hi == ed[i].hi; ++j) {
      if (neu[ed[j].e]) {
        if (n_n < 2) en[n_n] = ed[j].e;
        ++n_n;
      } else {
        ++n_d;
      }
    }
    if (n_n > 0 && n_d == 0) out.push_back({ed[i].lo, ed[i].hi, en[0], en[1], n_n != 2});
    i = j;
  }
  return out;
}

// A candidate whose two elements lie in one line / plane (unit normals equal
// to within 2^-23, FP32 resolution) has no dihedral angle: every point has
// the same signed distance to both, so the silhouette rule never holds for
// it.  Such candidates (the inside of a flat wall) stay out of the tree: a
// walker on the wall could otherwise prune none of them by its cone.
static bool flat_candidate(int dim, const float* verts, const int32_t* prims, const SilCand& c) {
  if (c.always || c.e0 < 0 || c.e1 < 0) return false;
  double n0[3] = {0, 0, 0}, n1[3] = {0, 0, 0};
  elem_normal(dim, verts, prims + (int64_t)c.e0 * dim, n0);
  elem_normal(dim, verts, prims + (int64_t)c.e1 * dim, n1);
  double d2 = 0.0;
  for (int a = 0; a < dim; ++a) d2 += (n0[a] - n1[a]) * (n0[a] - n1[a]);
  return d2 <= 0x1p-46;
}

static size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

// Normal cones of the silhouette tree: a cone (unit axis, half-angle)
// holding a set of unit normals; half-angles from pi/2 up are useless for
// pruning and stored as "full" (pi).
struct Cone {
  double a[3];
  double th;
};
static const double kFullCone = 3.14159265358979323846;

static Cone cone_merge(const Cone& c1, const Cone& c2) {
  if (c1.th >= kFullCone) return c1;
  if (c2.th >= kFullCone) return c2;
  double ca = c1.a[0] * c2.a[0] + c1.a[1] * c2.a[1] + c1.a[2] * c2.a[2];
  ca = std::min(1.0, std::max(-1.0, ca));
  const double al = std::acos(ca);
  if (al + c2.th <= c1.th) return c1;
  if (al + c1.th <= c2.th) return c2;
  Cone r;
  r.th = 0.5 * (al + c1.th + c2.th);
  if (r.th >= 0.5 * kFullCone - 1e-6) {
    r.a[0] = r.a[1] = r.a[2] = 0.0;
    r.th = kFullCone;
    return r;
  }
  // rotate c1's axis towards c2's by th - th1 (spherical interpolation)
  const double t = (r.th - c1.th) / al, sa = std::sin(al);
  const double w1 = std::sin((1.0 - t) * al) / sa, w2 = std::sin(t * al) / sa;
  double nn = 0.0;
  for (int k = 0; k < 3; ++k) {
    r.a[k] = w1 * c1.a[k] + w2 * c2.a[k];
    nn += r.a[k] * r.a[k];
  }
  nn = std::sqrt(nn);
  for (int k = 0; k < 3; ++k) r.a[k] /= nn;
  return r;
}

static bool fill_params(bvc_mixed m, const bvc_function* gfn, const bvc_neumann* h, const bvc_function* ffn,
                        WostParams& P) {
  P = WostParams{};
  P.Gd = m->dir->dev;
  P.Ga = m->whole->dev;
  if (m->neu) P.Gn = m->neu->dev;
  // one status block for the solve: debug bounds flags of the parts land in
  // the whole boundary's
  P.Gd.stats = P.Ga.stats;
  P.Gn.stats = P.Ga.stats;
  P.has_neu = m->neu != nullptr;
  P.S = m->sil;
  P.neu_local = m->neu_local;
  P.dir_ids = m->dir_ids;
  P.nmeas = m->nmeas;
  P.neu_q = m->neu_q;
  {
    double d2 = 0.0;
    for (int a = 0; a < m->dim; ++a) d2 += ((double)m->whole->hi[a] - m->whole->lo[a]) * (m->whole->hi[a] - m->whole->lo[a]);
    P.escape = (float)(4.0 * std::sqrt(d2));
  }
  P.stats = m->whole->dev.stats;
  const int D = m->dim;
  if (!make_dev_function(gfn, D, &P.g) || !make_dev_function(ffn, D, &P.f)) return false;
  if (h != nullptr) {
    if (!make_dev_function(&h->value, D, &P.hv) || !make_dev_function(&h->potential, D, &P.hp)) return false;
  }
  return true;
}

static bool valid_walk(float eps, int32_t max_steps, int32_t walks) {
  return std::isfinite(eps) && eps > 0.0f && max_steps >= 1 && walks >= 1;
}
static bool valid_sigma(double sigma) { return std::isfinite(sigma) && sigma >= 0.0; }

}  // namespace bvc

using namespace bvc;

static bvc_status bvc_mixed_create_impl(int32_t dim, const float* verts, int64_t n_verts, const int32_t* prims,
                                       int64_t n_prims, const uint8_t* neumann, bvc_stream stream, bvc_mixed* out) {
  if (out == nullptr) return BVC_ERR_INVALID_ARG;
  *out = nullptr;
  if ((dim != 2 && dim != 3) || verts == nullptr || prims == nullptr || neumann == nullptr || n_verts <= 0 ||
      n_prims <= 0)
    return BVC_ERR_INVALID_ARG;
  std::vector<int32_t> fd, fn;
  std::vector<int32_t> dir_ids, neu_local(n_prims, -1);
  for (int64_t e = 0; e < n_prims; ++e) {
    std::vector<int32_t>& dst = neumann[e] ? fn : fd;
    if (neumann[e]) neu_local[e] = (int32_t)(fn.size() / dim);
    else dir_ids.push_back((int32_t)e);
    for (int a = 0; a < dim; ++a) dst.push_back(prims[e * dim + a]);
  }
  const int64_t nd = (int64_t)fd.size() / dim, nn = (int64_t)fn.size() / dim;
  if (nd == 0) return BVC_ERR_INVALID_ARG;
  bvc_mixed m = new bvc_mixed_s();
  m->dim = dim;
  m->n_dir = nd;
  m->n_neu = nn;
  auto fail = [&](bvc_status st) {
    if (m->whole) bvc_geometry_destroy(m->whole);
    if (m->dir) bvc_geometry_destroy(m->dir);
    if (m->neu) bvc_geometry_destroy(m->neu);
    if (m->arena) cudaFree(m->arena);
    delete m;
    return st;
  };
  bvc_status st = bvc_geometry_create(dim, verts, n_verts, prims, n_prims, stream, &m->whole);
  if (st != BVC_OK) return fail(st);
  st = bvc_geometry_create(dim, verts, n_verts, fd.data(), nd, stream, &m->dir);
  if (st != BVC_OK) return fail(st);
  if (nn > 0) {
    st = bvc_geometry_create(dim, verts, n_verts, fn.data(), nn, stream, &m->neu);
    if (st != BVC_OK) return fail(st);
  }
  m->dir_measure = m->dir->measure;
  m->neu_measure = m->neu ? m->neu->measure : 0.0;
  // subtree measures of the Neumann tree (the same deterministic build as
  // the Neumann geometry's), for the area sampling of the Neumann term
  std::vector<float2> nmeas;
  std::vector<int32_t> nq;
  if (nn > 0) {
    std::vector<float4> nnodes, nprims;
    std::vector<int32_t> nids;
    const int64_t nnod = build_bvh(dim, verts, fn.data(), nn, nnodes, nprims, nids);
    nq.assign(nn, 0);
    for (int64_t q = 0; q < nn; ++q) nq[nids[q]] = (int32_t)q;
    const int per = dim == 2 ? 3 : 4;
    std::vector<double> em(nn);
    for (int64_t q = 0; q < nn; ++q) {
      double nrm_[3];
      em[q] = elem_normal(dim, verts, fn.data() + (int64_t)nids[q] * dim, nrm_);
    }
    std::vector<double> sub(nnod, -1.0);
    nmeas.assign(nnod, make_float2(0.0f, 0.0f));
    // children always follow their parent in the node array, so a reverse
    // sweep sees every child's total before its parent
    for (int64_t i = nnod - 1; i >= 0; --i) {
      const float4 c = nnodes[i * per + per - 1];
      int32_t ch[2];
      std::memcpy(&ch[0], &c.x, 4);
      std::memcpy(&ch[1], &c.y, 4);
      double w[2];
      for (int k = 0; k < 2; ++k) {
        if (ch[k] >= 0) {
          w[k] = sub[ch[k]];
        } else {
          const int32_t enc = ~ch[k];
          const int32_t first = enc >> 4, count = enc & 15;
          w[k] = 0.0;
          for (int32_t q = first; q < first + count; ++q) w[k] += em[q];
        }
      }
      sub[i] = w[0] + w[1];
      nmeas[i] = make_float2((float)w[0], (float)w[1]);
    }
  }
  // silhouette candidates and their tree
  std::vector<SilCand> cand = silhouette_candidates(dim, n_verts, prims, n_prims, neumann);
  m->n_sil = (int64_t)cand.size();
  cand.erase(std::remove_if(cand.begin(), cand.end(),
                            [&](const SilCand& c) { return flat_candidate(dim, verts, prims, c); }),
             cand.end());
  const int64_t ns = (int64_t)cand.size();
  std::vector<float4> snodes, sprims_unused, sprims;
  std::vector<int32_t> ids;
  if (ns > 0) {
    std::vector<int32_t> Fs((size_t)ns * dim);
    for (int64_t i = 0; i < ns; ++i) {
      Fs[i * dim] = cand[i].a;
      for (int a = 1; a < dim; ++a) Fs[i * dim + a] = cand[i].b;
    }
    build_bvh(dim, verts, Fs.data(), ns, snodes, sprims_unused, ids);
    const int per = dim == 2 ? 2 : 4;
    sprims.assign((size_t)ns * per, make_float4(0, 0, 0, 0));
    for (int64_t q = 0; q < ns; ++q) {
      const SilCand& c = cand[ids[q]];
      double n0[3] = {0, 0, 0}, n1[3] = {0, 0, 0};
      if (c.e0 >= 0 && !c.always) elem_normal(dim, verts, prims + (int64_t)c.e0 * dim, n0);
      if (c.e1 >= 0 && !c.always) elem_normal(dim, verts, prims + (int64_t)c.e1 * dim, n1);
      const float* va = verts + (int64_t)c.a * dim;
      const float* vb = verts + (int64_t)c.b * dim;
      if (dim == 2) {
        sprims[2 * q] = make_float4(va[0], va[1], (float)n0[0], (float)n0[1]);
        sprims[2 * q + 1] = make_float4((float)n1[0], (float)n1[1], c.always ? 1.0f : 0.0f, 0.0f);
      } else {
        const float abx = vb[0] - va[0], aby = vb[1] - va[1], abz = vb[2] - va[2];
        const float den = abx * abx + aby * aby + abz * abz;
        sprims[4 * q] = make_float4(va[0], va[1], va[2], c.always ? 1.0f : 0.0f);
        sprims[4 * q + 1] = make_float4(abx, aby, abz, den > 0.0f ? 1.0f / den : 0.0f);
        sprims[4 * q + 2] = make_float4((float)n0[0], (float)n0[1], (float)n0[2], 0.0f);
        sprims[4 * q + 3] = make_float4((float)n1[0], (float)n1[1], (float)n1[2], 0.0f);
      }
    }
  }
  m->n_sil_nodes = ns > 0 ? (int64_t)snodes.size() / (dim == 2 ? 3 : 4) : 0;
  // per node and child, the cone of the normals of the candidates below
  std::vector<float4> scones((size_t)m->n_sil_nodes * 2, make_float4(0, 0, 0, -1.0f));
  if (ns > 0) {
    const int per = dim == 2 ? 3 : 4;
    auto cand_cone = [&](int64_t q) {
      const SilCand& c = cand[ids[q]];
      Cone r{{0, 0, 0}, kFullCone};
      if (c.always) return r;
      double n0[3] = {0, 0, 0}, n1[3] = {0, 0, 0};
      elem_normal(dim, verts, prims + (int64_t)c.e0 * dim, n0);
      elem_normal(dim, verts, prims + (int64_t)c.e1 * dim, n1);
      Cone c0{{n0[0], n0[1], n0[2]}, 0.0}, c1{{n1[0], n1[1], n1[2]}, 0.0};
      return cone_merge(c0, c1);
    };
    std::vector<Cone> sub(m->n_sil_nodes);
    for (int64_t i = m->n_sil_nodes - 1; i >= 0; --i) {
      const float4 cc = snodes[i * per + per - 1];
      int32_t ch[2];
      std::memcpy(&ch[0], &cc.x, 4);
      std::memcpy(&ch[1], &cc.y, 4);
      Cone k2[2];
      for (int k = 0; k < 2; ++k) {
        if (ch[k] >= 0) {
          k2[k] = sub[ch[k]];
        } else {
          const int32_t enc = ~ch[k];
          const int32_t first = enc >> 4, count = enc & 15;
          Cone r{{0, 0, 0}, -1.0};
          for (int32_t q = first; q < first + count; ++q) r = r.th < 0.0 ? cand_cone(q) : cone_merge(r, cand_cone(q));
          k2[k] = r.th < 0.0 ? Cone{{0, 0, 0}, 0.0} : r;
        }
        // (axis, cos theta) with a little slack for the FP32 normals and axis;
        // cos theta <= 0: no bound
        const double th = k2[k].th + 1e-4;
        scones[2 * i + k] = make_float4((float)k2[k].a[0], (float)k2[k].a[1], (float)k2[k].a[2],
                                        th >= 0.5 * kFullCone ? -1.0f : (float)std::cos(th));
      }
      sub[i] = cone_merge(k2[0], k2[1]);
    }
  }
  const size_t b_nodes = al256(snodes.size() * sizeof(float4)), b_prims = al256(sprims.size() * sizeof(float4));
  const size_t b_dir = al256((size_t)nd * 4), b_loc = al256((size_t)n_prims * 4), b_flag = al256((size_t)n_prims);
  const size_t b_nm = al256(nmeas.size() * sizeof(float2)), b_nq = al256(nq.size() * 4);
  const size_t b_cone = al256(scones.size() * sizeof(float4));
  // the Dirichlet offset boundary: displacements from the Dirichlet
  // elements alone (a vertex shared with a Neumann element moves along its
  // Dirichlet element's normal; Neumann elements are not moved)
  std::vector<uint8_t> fl(n_prims);
  for (int64_t e = 0; e < n_prims; ++e) fl[e] = neumann[e] ? 1 : 0;
  std::vector<double> dsp((size_t)n_verts * dim);
  offset_disp(dim, verts, n_verts, prims, n_prims, fl.data(), dsp.data());
  const size_t b_disp = al256(dsp.size() * sizeof(double));
  m->arena_bytes = b_nodes + b_prims + b_dir + b_loc + b_flag + b_nm + b_nq + b_cone + b_disp;
  if (cudaMallocAsync(&m->arena, m->arena_bytes, (cudaStream_t)stream) != cudaSuccess) {
    (void)cudaGetLastError();
    m->arena = nullptr;
    return fail(BVC_ERR_OOM);
  }
  char* base = (char*)m->arena;
  m->sil.nodes = (const float4*)base;
  m->sil.prims = (const float4*)(base += b_nodes);
  m->dir_ids = (const int32_t*)(base += b_prims);
  m->neu_local = (const int32_t*)(base += b_dir);
  m->flags = (const uint8_t*)(base += b_loc);
  m->nmeas = (const float2*)(base += b_flag);
  m->neu_q = (const int32_t*)(base += b_nm);
  m->sil.cones = (const float4*)(base += b_nq);
  m->disp = (const double*)(base += b_cone);
  m->sil.n = ns;
  m->sil.n_nodes = m->n_sil_nodes;
  m->sil.stats = m->whole->dev.stats;
  m->sil.tau = m->whole->dev.tau;
  m->sil.shrink2 = 1.0f;
  cudaStream_t s = (cudaStream_t)stream;
  bool ok = true;
  if (ns > 0) {
    ok = ok && cudaMemcpyAsync((void*)m->sil.nodes, snodes.data(), snodes.size() * sizeof(float4),
                               cudaMemcpyHostToDevice, s) == cudaSuccess;
    ok = ok && cudaMemcpyAsync((void*)m->sil.prims, sprims.data(), sprims.size() * sizeof(float4),
                               cudaMemcpyHostToDevice, s) == cudaSuccess;
  }
  ok = ok && cudaMemcpyAsync((void*)m->dir_ids, dir_ids.data(), (size_t)nd * 4, cudaMemcpyHostToDevice, s) ==
                 cudaSuccess;
  ok = ok && cudaMemcpyAsync((void*)m->neu_local, neu_local.data(), (size_t)n_prims * 4, cudaMemcpyHostToDevice,
                             s) == cudaSuccess;
  ok = ok && cudaMemcpyAsync((void*)m->flags, fl.data(), (size_t)n_prims, cudaMemcpyHostToDevice, s) == cudaSuccess;
  ok = ok && cudaMemcpyAsync((void*)m->disp, dsp.data(), dsp.size() * 8, cudaMemcpyHostToDevice, s) == cudaSuccess;
  if (!nmeas.empty())
    ok = ok && cudaMemcpyAsync((void*)m->nmeas, nmeas.data(), nmeas.size() * sizeof(float2), cudaMemcpyHostToDevice,
                               s) == cudaSuccess;
  if (!nq.empty())
    ok = ok && cudaMemcpyAsync((void*)m->neu_q, nq.data(), nq.size() * 4, cudaMemcpyHostToDevice, s) == cudaSuccess;
  if (!scones.empty())
    ok = ok && cudaMemcpyAsync((void*)m->sil.cones, scones.data(), scones.size() * sizeof(float4),
                               cudaMemcpyHostToDevice, s) == cudaSuccess;
  if (!ok) {
    (void)cudaGetLastError();
    return fail(BVC_ERR_CUDA);
  }
  *out = m;
  return BVC_OK;
}
extern "C" bvc_status bvc_mixed_create(int32_t dim, const float* verts, int64_t n_verts, const int32_t* prims,
                                       int64_t n_prims, const uint8_t* neumann, bvc_stream stream, bvc_mixed* out) {
  return bvc::note_status(bvc_mixed_create_impl(dim, verts, n_verts, prims, n_prims, neumann, stream, out));
}

static bvc_status bvc_mixed_destroy_impl(bvc_mixed m) {
  if (m == nullptr) return BVC_ERR_INVALID_ARG;
  bvc_status st = BVC_OK;
  if (bvc_geometry_destroy(m->whole) != BVC_OK) st = BVC_ERR_CUDA;
  if (bvc_geometry_destroy(m->dir) != BVC_OK) st = BVC_ERR_CUDA;
  if (m->neu && bvc_geometry_destroy(m->neu) != BVC_OK) st = BVC_ERR_CUDA;
  if (cudaFree(m->arena) != cudaSuccess) st = BVC_ERR_CUDA;
  delete m;
  return st;
}
extern "C" bvc_status bvc_mixed_destroy(bvc_mixed m) {
  return bvc::note_status(bvc_mixed_destroy_impl(m));
}

static bvc_status bvc_mixed_get_info_impl(bvc_mixed m, bvc_mixed_info* info) {
  if (m == nullptr || info == nullptr) return BVC_ERR_INVALID_ARG;
  info->dim = m->dim;
  info->n_dirichlet = m->n_dir;
  info->n_neumann = m->n_neu;
  info->n_silhouette = m->n_sil;
  info->n_silhouette_tree = m->sil.n;
  info->dirichlet_measure = m->dir_measure;
  info->neumann_measure = m->neu_measure;
  info->device_bytes = m->arena_bytes;
  return BVC_OK;
}
extern "C" bvc_status bvc_mixed_get_info(bvc_mixed m, bvc_mixed_info* info) {
  return bvc::note_status(bvc_mixed_get_info_impl(m, info));
}

static bvc_status bvc_mixed_set_silhouette_gap_impl(bvc_mixed m, double gap) {
  if (m == nullptr || !(gap >= 0.0 && gap < 1.0)) return BVC_ERR_INVALID_ARG;
  m->sil.shrink2 = (float)((1.0 - gap) * (1.0 - gap));
  return BVC_OK;
}
extern "C" bvc_status bvc_mixed_set_silhouette_gap(bvc_mixed m, double gap) {
  return bvc::note_status(bvc_mixed_set_silhouette_gap_impl(m, gap));
}

static bvc_status bvc_mixed_geometries_impl(bvc_mixed m, bvc_geometry* whole, bvc_geometry* dirichlet,
                                           bvc_geometry* neumann) {
  if (m == nullptr) return BVC_ERR_INVALID_ARG;
  if (whole) *whole = m->whole;
  if (dirichlet) *dirichlet = m->dir;
  if (neumann) *neumann = m->neu;
  return BVC_OK;
}
extern "C" bvc_status bvc_mixed_geometries(bvc_mixed m, bvc_geometry* whole, bvc_geometry* dirichlet,
                                           bvc_geometry* neumann) {
  return bvc::note_status(bvc_mixed_geometries_impl(m, whole, dirichlet, neumann));
}

static int small_grid(int64_t n) {
  int64_t g = (n + kWostBlock - 1) / kWostBlock;
  const int64_t cap = (int64_t)num_sms() * 8;
  if (g > cap) g = cap;
  return (int)(g > 0 ? g : 1);
}

static bvc_status bvc_mixed_query_impl(bvc_mixed m, const float* pts, int64_t n, float* d_dir, float* d_sil,
                                      bvc_stream stream) {
  if (m == nullptr || n < 0 || (n > 0 && pts == nullptr)) return BVC_ERR_INVALID_ARG;
  if (n == 0) return BVC_OK;
  cudaStream_t s = (cudaStream_t)stream;
  ProfScope ps("mixed_query", s);
  if (m->dim == 2)
    k_mixed_query<2><<<small_grid(n), kWostBlock, 0, s>>>(m->dir->dev, m->sil, pts, n, d_dir, d_sil);
  else
    k_mixed_query<3><<<small_grid(n), kWostBlock, 0, s>>>(m->dir->dev, m->sil, pts, n, d_dir, d_sil);
  BVC_LAUNCH_CHECK();
  return BVC_OK;
}
extern "C" bvc_status bvc_mixed_query(bvc_mixed m, const float* pts, int64_t n, float* d_dir, float* d_sil,
                                      bvc_stream stream) {
  return bvc::note_status(bvc_mixed_query_impl(m, pts, n, d_dir, d_sil, stream));
}

static bvc_status bvc_mixed_rays_impl(bvc_mixed m, const float* org, const float* dir, const int32_t* skip, int64_t n,
                                     float tmax, float* t, int32_t* elem, bvc_stream stream) {
  if (m == nullptr || n < 0 || !(tmax > 0.0f) ||
      (n > 0 && (org == nullptr || dir == nullptr || t == nullptr || elem == nullptr)))
    return BVC_ERR_INVALID_ARG;
  if (n == 0) return BVC_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const DevGeometry Gn = m->neu ? m->neu->dev : DevGeometry{};
  ProfScope ps("mixed_rays", s);
  if (m->dim == 2)
    k_mixed_rays<2><<<small_grid(n), kWostBlock, 0, s>>>(Gn, m->neu != nullptr, org, dir, skip, n, tmax, t, elem);
  else
    k_mixed_rays<3><<<small_grid(n), kWostBlock, 0, s>>>(Gn, m->neu != nullptr, org, dir, skip, n, tmax, t, elem);
  BVC_LAUNCH_CHECK();
  return BVC_OK;
}
extern "C" bvc_status bvc_mixed_rays(bvc_mixed m, const float* org, const float* dir, const int32_t* skip, int64_t n,
                                     float tmax, float* t, int32_t* elem, bvc_stream stream) {
  return bvc::note_status(bvc_mixed_rays_impl(m, org, dir, skip, n, tmax, t, elem, stream));
}

static bvc_status bvc_mixed_walk_impl(bvc_mixed m, const bvc_function* gfn, const bvc_neumann* h,
                                     const bvc_function* ffn, double sigma, const float* starts,
                                     const int32_t* start_elem, const float* nrm, int64_t n, int32_t walks, float eps,
                                     int32_t max_steps, uint64_t seed, uint64_t id_base, uint32_t tag, float* rec,
                                     int32_t* steps, int32_t* prim, unsigned long long* counter, bvc_stream stream) {
  if (m == nullptr || n < 0 || !valid_walk(eps, max_steps, walks) || !valid_sigma(sigma)) return BVC_ERR_INVALID_ARG;
  if (n == 0) return BVC_OK;
  if (starts == nullptr || rec == nullptr || counter == nullptr || (start_elem != nullptr && nrm == nullptr))
    return BVC_ERR_INVALID_ARG;
  WostParams P;
  if (!fill_params(m, gfn, h, ffn, P)) return BVC_ERR_INVALID_ARG;
  P.sqs = (float)std::sqrt(sigma);
  P.starts = starts;
  P.start_elem = start_elem;
  P.nrm = nrm;
  P.pt_stride = n;
  P.i0 = 0;
  P.W = walks;
  P.total = n * (int64_t)walks;
  P.wid0 = id_base;
  P.eps = eps;
  P.max_steps = max_steps;
  P.seed = seed;
  P.tag = tag;
  P.rec = rec;
  P.steps = steps;
  P.prim = prim;
  P.counter = counter;
  return launch_wost(m->dim, nrm != nullptr ? kRecGnW : kRecGradW, P, (cudaStream_t)stream);
}
extern "C" bvc_status bvc_mixed_walk(bvc_mixed m, const bvc_function* gfn, const bvc_neumann* h,
                                     const bvc_function* ffn, const float* starts, const int32_t* start_elem,
                                     const float* nrm, int64_t n, int32_t walks, float eps, int32_t max_steps,
                                     uint64_t seed, uint64_t id_base, uint32_t tag, float* rec, int32_t* steps,
                                     int32_t* prim, unsigned long long* counter, bvc_stream stream) {
  return bvc::note_status(bvc_mixed_walk_impl(m, gfn, h, ffn, 0.0, starts, start_elem, nrm, n, walks, eps, max_steps,
                                              seed, id_base, tag, rec, steps, prim, counter, stream));
}
extern "C" bvc_status bvc_mixed_walk_sigma(bvc_mixed m, const bvc_function* gfn, const bvc_neumann* h,
                                           const bvc_function* ffn, double sigma, const float* starts,
                                           const int32_t* start_elem, const float* nrm, int64_t n, int32_t walks,
                                           float eps, int32_t max_steps, uint64_t seed, uint64_t id_base,
                                           uint32_t tag, float* rec, int32_t* steps, int32_t* prim,
                                           unsigned long long* counter, bvc_stream stream) {
  return bvc::note_status(bvc_mixed_walk_impl(m, gfn, h, ffn, sigma, starts, start_elem, nrm, n, walks, eps,
                                              max_steps, seed, id_base, tag, rec, steps, prim, counter, stream));
}

// Workspace of the mixed cache: [0, 256) work counter, the samples' elements
// (int32[N]), then the chunk's walk records (2 planes).
static size_t mixed_head(int64_t N) { return 256 + al256((size_t)N * 4); }

static bvc_status bvc_mixed_cache_build_workspace_size_impl(bvc_mixed m, const bvc_cache_opts* opts, size_t* min_bytes,
                                                           size_t* full_bytes) {
  if (m == nullptr || opts == nullptr || opts->n_samples < 0 || opts->walks_per_sample < 1)
    return BVC_ERR_INVALID_ARG;
  const size_t per = (size_t)opts->walks_per_sample * 2 * sizeof(float);
  const size_t head = mixed_head(opts->n_samples) + 256;
  size_t src = 0;
  const int64_t ncand = (int64_t)opts->src_grid[0] * opts->src_grid[1] * (m->dim == 3 ? opts->src_grid[2] : 1);
  if (ncand > 0) bvc_sample_source_workspace_size(ncand, &src);
  const size_t mn = head + per, full = head + per * (size_t)opts->n_samples;
  if (min_bytes) *min_bytes = mn > src ? mn : src;
  if (full_bytes) *full_bytes = full > src ? full : src;
  return BVC_OK;
}
extern "C" bvc_status bvc_mixed_cache_build_workspace_size(bvc_mixed m, const bvc_cache_opts* opts, size_t* min_bytes,
                                                           size_t* full_bytes) {
  return bvc::note_status(bvc_mixed_cache_build_workspace_size_impl(m, opts, min_bytes, full_bytes));
}

static bvc_status bvc_mixed_cache_build_impl(bvc_mixed m, const bvc_function* gfn, const bvc_neumann* h,
                                            const bvc_function* ffn, const bvc_cache_opts* opts, bvc_cache* cache,
                                            void* workspace, size_t workspace_bytes, bvc_stream stream) {
  if (m == nullptr || opts == nullptr || cache == nullptr) return BVC_ERR_INVALID_ARG;
  const int D = m->dim;
  const int64_t N = opts->n_samples;
  const int32_t W = opts->walks_per_sample;
  if (cache->dim != D || cache->n != N || N < 1 || !valid_walk((float)opts->eps, opts->max_steps, W) ||
      !(opts->offset_l > 0.0) || cache->z == nullptr || cache->nrm == nullptr || cache->jac == nullptr ||
      cache->u_hat == nullptr ||
      cache->dudn_hat == nullptr || cache->packed == nullptr || workspace == nullptr)
    return BVC_ERR_INVALID_ARG;
  if (!valid_sigma(opts->sigma)) return BVC_ERR_INVALID_ARG;
  if (opts->clamp_c != 0.0) return BVC_ERR_UNSUPPORTED;
  const int64_t ncand = (int64_t)opts->src_grid[0] * opts->src_grid[1] * (D == 3 ? opts->src_grid[2] : 1);
  if (ncand != cache->n_src_cand || ncand < 0) return BVC_ERR_INVALID_ARG;
  WostParams P;
  if (!fill_params(m, gfn, h, ffn, P)) return BVC_ERR_INVALID_ARG;
  const size_t head = mixed_head(N) + 256;
  const size_t per = (size_t)W * 2 * sizeof(float);
  if (workspace_bytes < head + per) return BVC_ERR_WORKSPACE;
  int64_t chunk = (int64_t)((workspace_bytes - head) / per);
  if (chunk > N) chunk = N;
  cudaStream_t s = (cudaStream_t)stream;
  P.sqs = (float)std::sqrt(opts->sigma);
  cache->sigma = opts->sigma;
  cache->clamp_c = 0.0;
  cache->bnd_measure = m->whole->measure;
  int32_t* elem = (int32_t*)((char*)workspace + 256);
  bvc_status st = launch_sample_boundary(m->whole, N, opts->offset_l, opts->seed, cache->z, cache->nrm, cache->jac,
                                         elem, N, s, nullptr, m->flags, m->disp);
  if (st != BVC_OK) return st;
  P.starts = cache->z;
  P.start_elem = elem;
  P.nrm = cache->nrm;
  P.pt_stride = N;
  P.W = W;
  P.eps = (float)opts->eps;
  P.max_steps = opts->max_steps;
  P.seed = opts->seed;
  P.tag = 0;
  P.counter = (unsigned long long*)workspace;
  P.rec = (float*)((char*)workspace + head);
  for (int64_t i0 = 0; i0 < N; i0 += chunk) {
    const int64_t c = (N - i0) < chunk ? (N - i0) : chunk;
    P.i0 = i0;
    P.total = c * (int64_t)W;
    P.wid0 = opts->walk_id_base + (uint64_t)i0 * (uint64_t)W;
    st = launch_wost(D, kRecGnW, P, s);
    if (st != BVC_OK) return st;
    ReduceParams R{};
    R.rec = P.rec;
    R.n = c;
    R.W = W;
    R.planes = 2;
    R.stride = P.total;
    R.mode = 0;
    R.out[0] = cache->u_hat + i0;
    R.out[1] = cache->dudn_hat + i0;
    st = launch_reduce(R, s);
    if (st != BVC_OK) return st;
  }
  if (ncand > 0) {
    st = opts->reuse_sources ? bvc_source_reweight(m->whole, ffn, cache, s)
                             : bvc_sample_source(m->whole, ffn, opts->src_grid, opts->seed, 0.0, cache, workspace,
                                                 workspace_bytes, stream);
    if (st != BVC_OK) return st;
  }
  return bvc_cache_pack(cache, stream);
}
extern "C" bvc_status bvc_mixed_cache_build(bvc_mixed m, const bvc_function* gfn, const bvc_neumann* h,
                                            const bvc_function* ffn, const bvc_cache_opts* opts, bvc_cache* cache,
                                            void* workspace, size_t workspace_bytes, bvc_stream stream) {
  return bvc::note_status(bvc_mixed_cache_build_impl(m, gfn, h, ffn, opts, cache, workspace, workspace_bytes, stream));
}

static bvc_status wost_estimate_impl(bvc_mixed m, const bvc_function* gfn, const bvc_neumann* h,
                                    const bvc_function* ffn, double sigma, bvc_eval_state* state, int32_t walks,
                                    float eps, int32_t max_steps, uint64_t seed, uint64_t id_base, void* workspace,
                                    size_t workspace_bytes, bvc_stream stream) {
  if (m == nullptr || state == nullptr || state->dim != m->dim || state->m < 0 || state->counts == nullptr ||
      !valid_walk(eps, max_steps, walks) || !valid_sigma(sigma))
    return BVC_ERR_INVALID_ARG;
  const int64_t M = state->m;
  if (M > 0 && (state->x == nullptr || state->u_bnd == nullptr || workspace == nullptr)) return BVC_ERR_INVALID_ARG;
  const int D = m->dim;
  WostParams P;
  if (!fill_params(m, gfn, h, ffn, P)) return BVC_ERR_INVALID_ARG;
  P.sqs = (float)std::sqrt(sigma);
  cudaStream_t s = (cudaStream_t)stream;
  if (M > 0) {
    const size_t per = (size_t)walks * (1 + D) * sizeof(float);
    if (workspace_bytes < 512 + per) return BVC_ERR_WORKSPACE;
    int64_t chunk = (int64_t)((workspace_bytes - 512) / per);
    if (chunk > M) chunk = M;
    P.starts = state->x;
    P.pt_stride = M;
    P.W = walks;
    P.eps = eps;
    P.max_steps = max_steps;
    P.seed = seed;
    P.tag = 3;
    P.counter = (unsigned long long*)workspace;
    P.rec = (float*)((char*)workspace + 256);
    const bool grad = state->grad_bnd != nullptr;
    for (int64_t i0 = 0; i0 < M; i0 += chunk) {
      const int64_t c = (M - i0) < chunk ? (M - i0) : chunk;
      P.i0 = i0;
      P.total = c * (int64_t)walks;
      P.wid0 = id_base + (uint64_t)i0 * (uint64_t)walks;
      bvc_status st = launch_wost(D, kRecGradW, P, s);
      if (st != BVC_OK) return st;
      ReduceParams R{};
      R.rec = P.rec;
      R.n = c;
      R.W = walks;
      R.planes = grad ? 1 + D : 1;
      R.stride = P.total;
      R.mode = 1;
      R.out[0] = state->u_bnd + i0;
      if (grad)
        for (int a = 0; a < D; ++a) R.out[1 + a] = state->grad_bnd + (int64_t)a * M + i0;
      st = launch_reduce(R, s);
      if (st != BVC_OK) return st;
    }
  }
  {
    ProfScope ps("add_counts", s);
    k_mixed_add_count<<<1, 32, 0, s>>>(state->counts, walks);
  }
  BVC_LAUNCH_CHECK();
  return BVC_OK;
}
extern "C" bvc_status wost_estimate(bvc_mixed m, const bvc_function* gfn, const bvc_neumann* h,
                                    const bvc_function* ffn, bvc_eval_state* state, int32_t walks, float eps,
                                    int32_t max_steps, uint64_t seed, uint64_t id_base, void* workspace,
                                    size_t workspace_bytes, bvc_stream stream) {
  return bvc::note_status(wost_estimate_impl(m, gfn, h, ffn, 0.0, state, walks, eps, max_steps, seed, id_base,
                                             workspace, workspace_bytes, stream));
}
extern "C" bvc_status wost_estimate_sigma(bvc_mixed m, const bvc_function* gfn, const bvc_neumann* h,
                                          const bvc_function* ffn, double sigma, bvc_eval_state* state, int32_t walks,
                                          float eps, int32_t max_steps, uint64_t seed, uint64_t id_base,
                                          void* workspace, size_t workspace_bytes, bvc_stream stream) {
  return bvc::note_status(wost_estimate_impl(m, gfn, h, ffn, sigma, state, walks, eps, max_steps, seed, id_base,
                                             workspace, workspace_bytes, stream));
}
