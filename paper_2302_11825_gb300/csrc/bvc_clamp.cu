// bvc_clamp.cu -- the remainder of the clamped double-layer kernel
// (Sec. 3.3, Eq. 8-9): int [dG/dn - clamp_c(dG/dn)] u dz per evaluation point.
//
// dG/dn dz is the signed solid angle seen from the point x, so a direction w
// drawn uniformly (Philox id = point * n_dirs + j, word2 0, tag 4) and every
// crossing z of the ray x + t w with the sample surface gives the unbiased
// term sign(n.w) (1 - c/|dG/dn(x, z)|) u(z) / n_dirs wherever |dG/dn| > c;
// |dG/dn| = |n.w| / (2 pi t) (2D), |n.w| / (4 pi t^2) (3D), so rays stop at
// t = 1/(2 pi c) or (4 pi c)^(-1/2).  The sample surface is the offset
// boundary of a mesh at l (its vertices moved by -l m_v, Sec. 3.2: the
// surface the cache's samples lie on; l = 0 for a region's own boundary):
// the BVH's boxes are grown by l x max|m_v| and each element is tested at
// its moved position.  u at the crossings is estimated by walks on
// the domain (tag 5, walk id = crossing rank * walks + j, crossings ranked by
// point, direction and distance); the crossings are compacted in that order
// by a deterministic block scan.
#include <algorithm>
#include <cmath>

#include "bvc_device.cuh"
#include "bvc_internal.h"

namespace bvc {

constexpr int kMaxHits = 8;
constexpr int kRayBlock = 128;
constexpr int kRayStack = 48;

struct RayParams {
  DevGeometry S;  // sample surface
  float l;        // vertices moved by -l m_v
  const float* pts;
  int64_t m;
  int32_t n_dirs;
  uint64_t seed;
  float c, rmax;
  int64_t slots;  // m * n_dirs * kMaxHits
  float* hz;      // [D][slots] crossing points
  float* hw;      // [slots] weights (0 = none)
  int64_t* bcount;
  int64_t* boff;
  int64_t nblocks;  // slot blocks of kRayBlock * kMaxHits
  float* zc;        // [D][slots] compacted crossings
  float* wc;        // [slots]
  int64_t* owner;   // [slots] point of each compacted crossing
  int64_t* n_hits;  // [1]
};

// Slab test of the ray against a box grown by l; true when it meets the box
// at some t in [0, rmax].
template <int D>
__device__ __forceinline__ bool ray_box(const float* lo, const float* hi, const float* o, const float* inv, float l,
                                        float rmax) {
  float t0 = 0.0f, t1 = rmax;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const float ta = (lo[a] - l - o[a]) * inv[a], tb = (hi[a] + l - o[a]) * inv[a];
    t0 = fmaxf(t0, fminf(ta, tb));
    t1 = fminf(t1, fmaxf(ta, tb));
  }
  return t0 <= t1;
}

template <int D>
__global__ void __launch_bounds__(kRayBlock) k_rays(const RayParams R) {
  const int64_t q = blockIdx.x * (int64_t)kRayBlock + threadIdx.x;  // point * n_dirs + direction
  const int64_t nq = R.m * (int64_t)R.n_dirs;
  float th[kMaxHits], tn[kMaxHits];
  int nh = 0;
  float x[D], om[D], inv[D];
  if (q < nq) {
    const int64_t p = q / R.n_dirs;
#pragma unroll
    for (int a = 0; a < D; ++a) x[a] = R.pts[a * R.m + p];
    const U4 r = philox_draw(R.seed, (uint64_t)q, 0u, 4u);
    const float u0 = u01f(r.x);
    if (D == 2) {
      float sn, cs;
      sincospif(2.0f * u0, &sn, &cs);
      om[0] = cs;
      om[D - 1] = sn;
    } else {
      const float u1 = u01f(r.y);
      const float zc = 1.0f - 2.0f * u0, st = 2.0f * sqrtf(u0 * (1.0f - u0));
      float sn, cs;
      sincospif(2.0f * u1, &sn, &cs);
      om[0] = st * cs;
      om[1] = st * sn;
      om[D - 1] = zc;
    }
#pragma unroll
    for (int a = 0; a < D; ++a) inv[a] = 1.0f / om[a];
    int stk[kRayStack];
    int sp = 0, node = 0;
    const DevGeometry& G = R.S;
    for (;;) {
      int32_t ch[2];
      bool hit[2];
      if (dbg_bad(G, node < 0 || node >= G.n_nodes)) break;
      if (D == 2) {
        const float4 L = __ldg(&G.nodes[3 * node]), Rb = __ldg(&G.nodes[3 * node + 1]);
        const float4 Cc = __ldg(&G.nodes[3 * node + 2]);
        const float lo0[2] = {L.x, L.y}, hi0[2] = {L.z, L.w}, lo1[2] = {Rb.x, Rb.y}, hi1[2] = {Rb.z, Rb.w};
        hit[0] = ray_box<2>(lo0, hi0, x, inv, R.l * G.reach, R.rmax);
        hit[1] = ray_box<2>(lo1, hi1, x, inv, R.l * G.reach, R.rmax);
        ch[0] = __float_as_int(Cc.x);
        ch[1] = __float_as_int(Cc.y);
      } else {
        const float4 a = __ldg(&G.nodes[4 * node]), b = __ldg(&G.nodes[4 * node + 1]);
        const float4 c = __ldg(&G.nodes[4 * node + 2]), e = __ldg(&G.nodes[4 * node + 3]);
        const float lo0[3] = {a.x, a.y, a.z}, hi0[3] = {a.w, b.x, b.y};
        const float lo1[3] = {b.z, b.w, c.x}, hi1[3] = {c.y, c.z, c.w};
        hit[0] = ray_box<3>(lo0, hi0, x, inv, R.l * G.reach, R.rmax);
        hit[1] = ray_box<3>(lo1, hi1, x, inv, R.l * G.reach, R.rmax);
        ch[0] = __float_as_int(e.x);
        ch[1] = __float_as_int(e.y);
      }
      for (int k = 0; k < 2; ++k) {
        if (!hit[k]) continue;
        if (ch[k] >= 0) {
          if (sp < kRayStack)
            stk[sp++] = ch[k];
          else
            dbg_bad(G, true);
          continue;
        }
        const int32_t enc = ~ch[k];
        const int32_t first = enc >> 4, count = enc & 15;
        if (dbg_bad(G, first < 0 || (int64_t)first + count > G.n_prims)) continue;
        for (int32_t pq = first; pq < first + count; ++pq) {
          float t = -1.0f, nw = 0.0f;
          if (D == 2) {
            float4 S = __ldg(&G.prims[2 * pq]);
            if (R.l != 0.0f) {  // the moved segment: its vertices minus l m_v
              const int32_t* f = G.idx + 2 * __float_as_int(__ldg(&G.prims[2 * pq + 1]).y);
              const float a0 = G.verts[2 * f[0]] - R.l * (float)G.disp[2 * f[0]];
              const float a1 = G.verts[2 * f[0] + 1] - R.l * (float)G.disp[2 * f[0] + 1];
              const float b0 = G.verts[2 * f[1]] - R.l * (float)G.disp[2 * f[1]];
              const float b1 = G.verts[2 * f[1] + 1] - R.l * (float)G.disp[2 * f[1] + 1];
              S = make_float4(a0, a1, b0 - a0, b1 - a1);
            }
            const float len = sqrtf(fmaf(S.w, S.w, S.z * S.z));
            const float nx = S.w / len, ny = -S.z / len;  // outward normal of a counter-clockwise polygon
            const float ax = S.x - x[0], ay = S.y - x[1];
            const float den = om[0] * S.w - om[D - 1] * S.z;
            if (den != 0.0f) {
              const float tt = (ax * S.w - ay * S.z) / den, ss = (ax * om[D - 1] - ay * om[0]) / den;
              if (ss >= 0.0f && ss <= 1.0f) t = tt;
            }
            nw = nx * om[0] + ny * om[D - 1];
          } else {
            float4 A = __ldg(&G.prims[3 * pq]), B = __ldg(&G.prims[3 * pq + 1]), Cq = __ldg(&G.prims[3 * pq + 2]);
            if (R.l != 0.0f) {  // the moved triangle: its vertices minus l m_v
              const int32_t* f = G.idx + 3 * __float_as_int(A.w);
              float P[3][3];
#pragma unroll
              for (int k2 = 0; k2 < 3; ++k2)
#pragma unroll
                for (int a = 0; a < 3; ++a) P[k2][a] = G.verts[3 * f[k2] + a] - R.l * (float)G.disp[3 * f[k2] + a];
              A = make_float4(P[0][0], P[0][1], P[0][2], A.w);
              B = make_float4(P[1][0] - P[0][0], P[1][1] - P[0][1], P[1][2] - P[0][2], 0.0f);
              Cq = make_float4(P[2][0] - P[0][0], P[2][1] - P[0][1], P[2][2] - P[0][2], 0.0f);
            }
            const float e1[3] = {B.x, B.y, B.z}, e2[3] = {Cq.x, Cq.y, Cq.z};
            float n3[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
            const float nl = rsqrtf(fmaf(n3[2], n3[2], fmaf(n3[1], n3[1], n3[0] * n3[0])));
#pragma unroll
            for (int a = 0; a < 3; ++a) n3[a] *= nl;
            // Moller-Trumbore on the (moved) triangle
            const float tv[3] = {x[0] - A.x, x[1] - A.y, x[D - 1] - A.z};
            const float o3[3] = {om[0], om[1], om[D - 1]};
            const float pv[3] = {o3[1] * e2[2] - o3[2] * e2[1], o3[2] * e2[0] - o3[0] * e2[2],
                                 o3[0] * e2[1] - o3[1] * e2[0]};
            const float det = e1[0] * pv[0] + e1[1] * pv[1] + e1[2] * pv[2];
            if (det != 0.0f) {
              const float id = 1.0f / det;
              const float uu = (tv[0] * pv[0] + tv[1] * pv[1] + tv[2] * pv[2]) * id;
              if (uu >= 0.0f && uu <= 1.0f) {
                const float qv[3] = {tv[1] * e1[2] - tv[2] * e1[1], tv[2] * e1[0] - tv[0] * e1[2],
                                     tv[0] * e1[1] - tv[1] * e1[0]};
                const float vv = (o3[0] * qv[0] + o3[1] * qv[1] + o3[2] * qv[2]) * id;
                if (vv >= 0.0f && uu + vv <= 1.0f) t = (e2[0] * qv[0] + e2[1] * qv[1] + e2[2] * qv[2]) * id;
              }
            }
            nw = n3[0] * o3[0] + n3[1] * o3[1] + n3[2] * o3[2];
          }
          if (!(t > 0.0f) || t > R.rmax) continue;
          // insert by distance, keep the nearest kMaxHits
          int pos = nh;
          while (pos > 0 && th[pos - 1] > t) --pos;
          if (pos >= kMaxHits) continue;
          for (int k2 = (nh < kMaxHits ? nh : kMaxHits - 1); k2 > pos; --k2) {
            th[k2] = th[k2 - 1];
            tn[k2] = tn[k2 - 1];
          }
          th[pos] = t;
          tn[pos] = nw;
          if (nh < kMaxHits) ++nh;
        }
      }
      if (sp == 0) break;
      node = stk[--sp];
    }
  }
  // slots of this ray: weights and crossing points
  int keep = 0;
  for (int k = 0; k < kMaxHits; ++k) {
    float w = 0.0f;
    if (q < nq && k < nh) {
      const float gn = D == 2 ? fabsf(tn[k]) / (6.28318530717958648f * th[k])
                              : fabsf(tn[k]) / (12.5663706143591730f * th[k] * th[k]);
      if (gn > R.c) {
        w = (tn[k] > 0.0f ? 1.0f : -1.0f) * (1.0f - R.c / gn) / (float)R.n_dirs;
        const int64_t sl = q * kMaxHits + k;
#pragma unroll
        for (int a = 0; a < D; ++a) R.hz[a * R.slots + sl] = fmaf(th[k], om[a], x[a]);
      }
    }
    if (q < nq) R.hw[q * kMaxHits + k] = w;
    keep += w != 0.0f;
  }
  (void)keep;
}

// Per block of kRayBlock rays (kRayBlock * kMaxHits slots): kept crossings.
__global__ void __launch_bounds__(kRayBlock) k_hits_count(const RayParams R) {
  __shared__ int part[kRayBlock];
  int c = 0;
  for (int k = 0; k < kMaxHits; ++k) {
    const int64_t sl = (blockIdx.x * (int64_t)kRayBlock + threadIdx.x) * kMaxHits + k;
    if (sl < R.slots && R.hw[sl] != 0.0f) ++c;
  }
  part[threadIdx.x] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t s = 0;
    for (int i = 0; i < kRayBlock; ++i) s += part[i];
    R.bcount[blockIdx.x] = s;
  }
}

// Exclusive scan of the block counts (one block, fixed order) and the total.
__global__ void __launch_bounds__(1024) k_hits_scan(const RayParams R) {
  __shared__ int64_t part[1024];
  const int64_t nb = R.nblocks;
  const int64_t per = (nb + 1023) / 1024;
  const int64_t b0 = threadIdx.x * per, b1 = min64(nb, b0 + per);
  int64_t s = 0;
  for (int64_t b = b0; b < b1; ++b) s += R.bcount[b];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t acc = 0;
    for (int i = 0; i < 1024; ++i) {
      const int64_t v = part[i];
      part[i] = acc;
      acc += v;
    }
    *R.n_hits = acc;
  }
  __syncthreads();
  int64_t acc = part[threadIdx.x];
  for (int64_t b = b0; b < b1; ++b) {
    const int64_t v = R.bcount[b];
    R.boff[b] = acc;
    acc += v;
  }
}

// Stable compaction of the kept crossings (slot order within a block: ray,
// then distance).
template <int D>
__global__ void __launch_bounds__(kRayBlock) k_hits_scatter(const RayParams R) {
  __shared__ int part[kRayBlock];
  const int64_t q = blockIdx.x * (int64_t)kRayBlock + threadIdx.x;
  int c = 0;
  for (int k = 0; k < kMaxHits; ++k) {
    const int64_t sl = q * kMaxHits + k;
    if (sl < R.slots && R.hw[sl] != 0.0f) ++c;
  }
  part[threadIdx.x] = c;
  __syncthreads();
  int before = 0;
  for (int i = 0; i < (int)threadIdx.x; ++i) before += part[i];
  int64_t j = R.boff[blockIdx.x] + before;
  for (int k = 0; k < kMaxHits; ++k) {
    const int64_t sl = q * kMaxHits + k;
    if (sl >= R.slots || R.hw[sl] == 0.0f) continue;
#pragma unroll
    for (int a = 0; a < D; ++a) R.zc[a * R.slots + j] = R.hz[a * R.slots + sl];
    R.wc[j] = R.hw[sl];
    R.owner[j] = q / R.n_dirs;
    ++j;
  }
}

// u_corr[owner] += w * mean U over the crossing's walks (FP64 atomics).
__global__ void __launch_bounds__(256) k_corr_scatter(const float* __restrict__ rec, int64_t c, int32_t W,
                                                     const float* __restrict__ wc, const int64_t* __restrict__ owner,
                                                     int64_t h0, double* __restrict__ u_corr) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < c; r += nwarps) {
    double s = 0.0;
    for (int j = lane; j < W; j += 32) s += (double)rec[r * W + j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) atomicAdd(&u_corr[owner[h0 + r]], (double)wc[h0 + r] * s / (double)W);
  }
}

static size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace bvc

using namespace bvc;

namespace {
struct CorrLayout {
  size_t hz, hw, bcount, boff, zc, wc, owner, nh, walks, total;
};

CorrLayout corr_layout(int dim, int64_t m, int32_t n_dirs) {
  const int64_t slots = m * (int64_t)n_dirs * kMaxHits;
  const int64_t nb = (m * (int64_t)n_dirs + kRayBlock - 1) / kRayBlock;
  CorrLayout L{};
  size_t o = 0;
  L.hz = o;
  o += al256((size_t)slots * dim * 4);
  L.hw = o;
  o += al256((size_t)slots * 4);
  L.bcount = o;
  o += al256((size_t)nb * 8);
  L.boff = o;
  o += al256((size_t)nb * 8);
  L.zc = o;
  o += al256((size_t)slots * dim * 4);
  L.wc = o;
  o += al256((size_t)slots * 4);
  L.owner = o;
  o += al256((size_t)slots * 8);
  L.nh = o;
  o += 256;
  L.walks = o;
  L.total = o;
  return L;
}
}  // namespace

static bvc_status bvc_clamp_correction_workspace_size_impl(int32_t dim, int64_t m, int32_t n_dirs, int32_t walks,
                                                          size_t* min_bytes) {
  if ((dim != 2 && dim != 3) || m < 0 || n_dirs < 1 || walks < 1 || min_bytes == nullptr) return BVC_ERR_INVALID_ARG;
  size_t per = 0;
  if (wos_estimate_workspace_size(dim, 1, walks, &per, nullptr) != BVC_OK) return BVC_ERR_INVALID_ARG;
  *min_bytes = corr_layout(dim, m, n_dirs).total + per;
  return BVC_OK;
}
extern "C" bvc_status bvc_clamp_correction_workspace_size(int32_t dim, int64_t m, int32_t n_dirs, int32_t walks,
                                                          size_t* min_bytes) {
  return bvc::note_status(bvc_clamp_correction_workspace_size_impl(dim, m, n_dirs, walks, min_bytes));
}

static bvc_status bvc_clamp_correction_impl(bvc_geometry domain, bvc_geometry surface, double offset_l,
                                           const bvc_function* gfn, const bvc_function* ffn, double sigma,
                                           double clamp_c, const float* pts, int64_t m, int32_t n_dirs,
                                           int32_t walks, float eps, int32_t max_steps, uint64_t seed,
                                           double* u_corr, int64_t* n_hits, void* workspace, size_t workspace_bytes,
                                           bvc_stream stream) {
  if (domain == nullptr || surface == nullptr || surface->dim != domain->dim || !(offset_l >= 0.0) ||
      !(clamp_c > 0.0) || m < 0 || n_dirs < 1 || walks < 1 || (m > 0 && (pts == nullptr || u_corr == nullptr)) ||
      workspace == nullptr)
    return BVC_ERR_INVALID_ARG;
  const int D = domain->dim;
  size_t need = 0;
  bvc_status st = bvc_clamp_correction_workspace_size(D, m, n_dirs, walks, &need);
  if (st != BVC_OK) return st;
  if (workspace_bytes < need) return BVC_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  if (n_hits) *n_hits = 0;
  if (m == 0) return BVC_OK;
  BVC_CUDA_TRY(cudaMemsetAsync(u_corr, 0, (size_t)m * sizeof(double), s));
  const CorrLayout L = corr_layout(D, m, n_dirs);
  char* w = (char*)workspace;
  RayParams R{};
  R.S = surface->dev;
  R.l = (float)offset_l;
  R.pts = pts;
  R.m = m;
  R.n_dirs = n_dirs;
  R.seed = seed;
  R.c = (float)clamp_c;
  R.rmax = (float)(D == 2 ? 1.0 / (2.0 * M_PI * clamp_c) : std::sqrt(1.0 / (4.0 * M_PI * clamp_c)));
  R.slots = m * (int64_t)n_dirs * kMaxHits;
  R.hz = (float*)(w + L.hz);
  R.hw = (float*)(w + L.hw);
  R.bcount = (int64_t*)(w + L.bcount);
  R.boff = (int64_t*)(w + L.boff);
  R.zc = (float*)(w + L.zc);
  R.wc = (float*)(w + L.wc);
  R.owner = (int64_t*)(w + L.owner);
  R.n_hits = (int64_t*)(w + L.nh);
  R.nblocks = (m * (int64_t)n_dirs + kRayBlock - 1) / kRayBlock;
  {
    ProfScope ps("clamp_rays", s);
    if (D == 2)
      k_rays<2><<<(unsigned)R.nblocks, kRayBlock, 0, s>>>(R);
    else
      k_rays<3><<<(unsigned)R.nblocks, kRayBlock, 0, s>>>(R);
    k_hits_count<<<(unsigned)R.nblocks, kRayBlock, 0, s>>>(R);
    k_hits_scan<<<1, 1024, 0, s>>>(R);
    if (D == 2)
      k_hits_scatter<2><<<(unsigned)R.nblocks, kRayBlock, 0, s>>>(R);
    else
      k_hits_scatter<3><<<(unsigned)R.nblocks, kRayBlock, 0, s>>>(R);
    BVC_LAUNCH_CHECK();
  }
  int64_t H = 0;
  BVC_CUDA_TRY(cudaMemcpyAsync(&H, R.n_hits, sizeof(H), cudaMemcpyDeviceToHost, s));
  BVC_CUDA_TRY(cudaStreamSynchronize(s));
  if (n_hits) *n_hits = H;
  if (H == 0) return BVC_OK;
  // walks from the crossings, in chunks that fit the rest of the workspace;
  // the crossings are laid out as a [D][slots] point set, so each chunk is
  // a pointwise estimate on the range [h0, h0 + c)
  void* ws = w + L.walks;
  const size_t ws_bytes = workspace_bytes - L.walks;
  size_t per = 0;
  wos_estimate_workspace_size(D, 1, walks, &per, nullptr);
  per -= 512;  // per start (the head is counted once below)
  int64_t chunk = (int64_t)((ws_bytes - 512) / per);
  if (chunk < 1) return BVC_ERR_WORKSPACE;
  for (int64_t h0 = 0; h0 < H; h0 += chunk) {
    const int64_t c = std::min<int64_t>(chunk, H - h0);
    st = walk_points_u(domain, gfn, ffn, sigma, R.zc, R.slots, h0, c, walks, eps, max_steps, seed, 5u,
                       (uint64_t)h0 * (uint64_t)walks, ws, ws_bytes, s);
    if (st != BVC_OK) return st;
    const float* rec = walk_records_u(ws, c, D);
    int64_t blocks = (c * 32 + 255) / 256;
    const int64_t cap = (int64_t)num_sms() * 16;
    if (blocks > cap) blocks = cap;
    ProfScope ps("clamp_scatter", s);
    k_corr_scatter<<<(unsigned)blocks, 256, 0, s>>>(rec, c, walks, R.wc, R.owner, h0, u_corr);
    BVC_LAUNCH_CHECK();
  }
  return BVC_OK;
}
extern "C" bvc_status bvc_clamp_correction(bvc_geometry domain, bvc_geometry surface, double offset_l,
                                           const bvc_function* gfn, const bvc_function* ffn, double sigma,
                                           double clamp_c, const float* pts, int64_t m, int32_t n_dirs,
                                           int32_t walks, float eps, int32_t max_steps, uint64_t seed,
                                           double* u_corr, int64_t* n_hits, void* workspace, size_t workspace_bytes,
                                           bvc_stream stream) {
  return bvc::note_status(bvc_clamp_correction_impl(domain, surface, offset_l, gfn, ffn, sigma, clamp_c, pts, m, n_dirs, walks, eps, max_steps, seed, u_corr, n_hits, workspace, workspace_bytes, stream));
}
