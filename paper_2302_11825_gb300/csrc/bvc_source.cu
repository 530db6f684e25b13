// bvc_source.cu -- source samples (K4): jittered candidates over the
// bounding box, kept by the canonical FP32 crossing test (2D) or a winding
// number above 1/2 (3D) against the offset boundary (the mesh with its
// vertices moved to fl32(v - l m_v), Sec. 3.2: the region the cache's
// integral equation refers to), compacted in candidate order by a
// deterministic block scan.
#include <algorithm>
#include <cmath>

#include "bvc_device.cuh"
#include "bvc_internal.h"

namespace bvc {

constexpr int kSrcBlock = 256;
constexpr int kSegTile = 1024;

struct SrcParams {
  DevGeometry G;
  double l;           // offset of the region's boundary (0: the mesh itself)
  DevFunction f;
  int32_t G0, G1, G2;
  uint64_t seed;
  double lo0, lo1, lo2, h0, h1, h2, box;
  int64_t ncand;
  float* yc;          // [dim][ncand] candidate positions (workspace)
  uint8_t* flag;      // [ncand] (workspace)
  int64_t* bcount;    // [nblocks] (workspace)
  int64_t* boff;      // [nblocks] (workspace)
  float* theta;       // [slices][ncand] 3D partial angle sums (workspace)
  int32_t slices;     // 3D: triangle slices per candidate
  float* src_y;       // [dim][ncand]
  double* src_c;      // [ncand]
  int64_t* n_src;     // [1]
  int64_t nblocks;
};

// Coordinate k of the offset boundary's vertex list: fl32(v - l m) in FP64.
__device__ __forceinline__ float moved_vertex(const SrcParams& S, int64_t k) {
  return S.l == 0.0 ? S.G.verts[k] : __double2float_rn(__dsub_rn((double)S.G.verts[k], __dmul_rn(S.l, S.G.disp[k])));
}

// Candidate position (FP64, rounded to FP32) and the crossing-number test
// against every segment, staged through shared memory.
__global__ void __launch_bounds__(kSrcBlock) k_src_classify(const SrcParams S) {
  __shared__ float4 seg[kSegTile];
  const int64_t c = blockIdx.x * (int64_t)kSrcBlock + threadIdx.x;
  float px = 0.0f, py = 0.0f;
  if (c < S.ncand) {
    const U4 r = philox_draw(S.seed, (uint64_t)c, 0u, 2u);
    const int64_t c0 = c % S.G0, c1 = c / S.G0;
    const double y0 = __dadd_rn(S.lo0, __dmul_rn(__dadd_rn((double)c0, u01d(r.x)), S.h0));
    const double y1 = __dadd_rn(S.lo1, __dmul_rn(__dadd_rn((double)c1, u01d(r.y)), S.h1));
    px = __double2float_rn(y0);
    py = __double2float_rn(y1);
    S.yc[c] = px;
    S.yc[S.ncand + c] = py;
  }
  int par = 0;
  const int64_t np = S.G.n_prims;
  for (int64_t base = 0; base < np; base += kSegTile) {
    __syncthreads();
    for (int q = threadIdx.x; q < kSegTile && base + q < np; q += kSrcBlock) {
      const int32_t* f = S.G.idx + 2 * (base + q);
      seg[q] = make_float4(moved_vertex(S, 2 * f[0]), moved_vertex(S, 2 * f[0] + 1), moved_vertex(S, 2 * f[1]),
                           moved_vertex(S, 2 * f[1] + 1));
    }
    __syncthreads();
    const int cnt = (int)min64(kSegTile, np - base);
    for (int q = 0; q < cnt; ++q) {
      const float4 s = seg[q];
      if ((s.y > py) != (s.w > py)) {
        const float t = __fdiv_rn(__fsub_rn(py, s.y), __fsub_rn(s.w, s.y));
        const float xi = __fmaf_rn(t, __fsub_rn(s.z, s.x), s.x);
        if (px < xi) par ^= 1;
      }
    }
  }
  const int keep = (c < S.ncand) ? par : 0;
  if (c < S.ncand) S.flag[c] = (uint8_t)keep;
  const int cnt = __syncthreads_count(keep);
  if (threadIdx.x == 0) S.bcount[blockIdx.x] = cnt;
}

// Exclusive scan of the block counts (one block, fixed order).
__global__ void __launch_bounds__(1024) k_src_scan(const SrcParams S) {
  __shared__ int64_t part[1024];
  const int64_t nb = S.nblocks;
  const int64_t per = (nb + 1023) / 1024;
  const int64_t b0 = threadIdx.x * per, b1 = min64(nb, b0 + per);
  int64_t s = 0;
  for (int64_t b = b0; b < b1; ++b) s += S.bcount[b];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t acc = 0;
    for (int q = 0; q < 1024; ++q) {
      const int64_t v = part[q];
      part[q] = acc;
      acc += v;
    }
    *S.n_src = acc;
  }
  __syncthreads();
  int64_t acc = part[threadIdx.x];
  for (int64_t b = b0; b < b1; ++b) {
    S.boff[b] = acc;
    acc += S.bcount[b];
  }
}

// 3D: candidate position as in 2D, kept when the generalized winding number
// of the triangle mesh (Jacobson et al. 2013) is above 1/2.  Each triangle
// subtends the solid angle 2 theta, theta = arg(den + i num) with
// num = A.(BxC), den = |A||B||C| + (A.B)|C| + (A.C)|B| + (B.C)|A| (Van
// Oosterom and Strackee 1983), so w = sum theta / (2 pi).  Rather than one
// arctangent per triangle, the kernel multiplies the complex numbers
// (den + i num) -- scaled to unit size -- into a running product and counts
// the product's crossings of the negative real axis (each factor turns it
// by |theta| < pi, counter-clockwise when num > 0); then
// sum theta = 2 pi crossings + arg(product), one arctangent per candidate.
// Triangles are staged through shared memory.  It is 1 inside a closed
// outward-wound surface and counts overlapping or nested shells with their
// orientation (an unrepaired self-intersecting boundary is classified the
// same way).
// The triangles are split into S.slices contiguous ranges (blockIdx.y), so
// that enough blocks run for the latency of each thread's serial product to
// be hidden; every slice writes its partial angle sum and k_src_flag3d adds
// the slices in a fixed order.
constexpr int kTriTile = 256;
constexpr int kMaxSlices = 16;

// Approximate reciprocal (MUFU.RCP): the factors are only rescaled by it.
__device__ __forceinline__ float rcp_fast(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__global__ void __launch_bounds__(kSrcBlock) k_src_classify3d(const SrcParams S) {
  __shared__ float4 tri[3][kTriTile];
  const int64_t c = blockIdx.x * (int64_t)kSrcBlock + threadIdx.x;
  const int slice = blockIdx.y;
  float p[3] = {0.0f, 0.0f, 0.0f};
  if (c < S.ncand) {
    const U4 r = philox_draw(S.seed, (uint64_t)c, 0u, 2u);
    const int64_t ci[3] = {c % S.G0, (c / S.G0) % S.G1, c / ((int64_t)S.G0 * S.G1)};
    const double lo[3] = {S.lo0, S.lo1, S.lo2}, h[3] = {S.h0, S.h1, S.h2};
    const double u[3] = {u01d(r.x), u01d(r.y), u01d(r.z)};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      p[a] = __double2float_rn(__dadd_rn(lo[a], __dmul_rn(__dadd_rn((double)ci[a], u[a]), h[a])));
      if (slice == 0) S.yc[a * S.ncand + c] = p[a];
    }
  }
  float zr = 1.0f, zi = 0.0f;
  int crossings = 0;
  const int64_t per = (S.G.n_prims + S.slices - 1) / S.slices;
  const int64_t t0 = slice * per, np = min64(S.G.n_prims, t0 + per);
  for (int64_t base = t0; base < np; base += kTriTile) {
    __syncthreads();
    for (int q = threadIdx.x; q < kTriTile && base + q < np; q += kSrcBlock) {
      const int32_t* f = S.G.idx + 3 * (base + q);
#pragma unroll
      for (int v = 0; v < 3; ++v)
        tri[v][q] = make_float4(moved_vertex(S, 3 * f[v]), moved_vertex(S, 3 * f[v] + 1),
                                moved_vertex(S, 3 * f[v] + 2), 0.0f);
    }
    __syncthreads();
    const int cnt = (int)min64(kTriTile, np - base);
    // blocks of 16 triangles, the product renormalised after each block
    // (|factor| lies in [1, sqrt 2]); a degenerate factor (the point on a
    // triangle's edge) is replaced by 1
    for (int q0 = 0; q0 < cnt; q0 += 16) {
#pragma unroll 4
      for (int q = q0; q < q0 + 16; ++q) {
        if (q >= cnt) break;
        const float4 ta = tri[0][q], tb = tri[1][q], tc = tri[2][q];
        const float ax = ta.x - p[0], ay = ta.y - p[1], az = ta.z - p[2];
        const float bx = tb.x - p[0], by = tb.y - p[1], bz = tb.z - p[2];
        const float cx = tc.x - p[0], cy = tc.y - p[1], cz = tc.z - p[2];
        const float a2 = fmaf(az, az, fmaf(ay, ay, ax * ax));
        const float b2 = fmaf(bz, bz, fmaf(by, by, bx * bx));
        const float c2 = fmaf(cz, cz, fmaf(cy, cy, cx * cx));
        const float la = a2 * rsqrtf(a2), lb = b2 * rsqrtf(b2), lc = c2 * rsqrtf(c2);
        const float num = fmaf(az, fmaf(bx, cy, -by * cx), fmaf(ay, fmaf(bz, cx, -bx * cz), ax * fmaf(by, cz, -bz * cy)));
        const float ab = fmaf(az, bz, fmaf(ay, by, ax * bx)), ac = fmaf(az, cz, fmaf(ay, cy, ax * cx));
        const float bc = fmaf(bz, cz, fmaf(by, cy, bx * cx));
        const float den = fmaf(bc, la, fmaf(ac, lb, fmaf(ab, lc, la * lb * lc)));
        const float mm = fmaxf(fabsf(num), fabsf(den));
        const bool ok = mm > 0.0f && mm < 3.0e38f;
        const float sc = ok ? rcp_fast(mm) : 0.0f;
        const float wr = ok ? den * sc : 1.0f, wi = num * sc;
        const float nr = fmaf(zr, wr, -zi * wi), ni = fmaf(zr, wi, zi * wr);
        crossings += (zi >= 0.0f && ni < 0.0f && num > 0.0f) ? 1 : 0;
        crossings -= (zi < 0.0f && ni >= 0.0f && num < 0.0f) ? 1 : 0;
        zr = nr;
        zi = ni;
      }
      const float t = rsqrtf(fmaf(zi, zi, zr * zr));
      zr *= t;
      zi *= t;
    }
  }
  // this slice's sum of theta = 2 pi crossings + arg(product)
  if (c < S.ncand) S.theta[(int64_t)slice * S.ncand + c] = 6.28318530717958648f * (float)crossings + atan2f(zi, zr);
}

// w = sum theta / (2 pi) > 1/2; slices added in order.
__global__ void __launch_bounds__(kSrcBlock) k_src_flag3d(const SrcParams S) {
  const int64_t c = blockIdx.x * (int64_t)kSrcBlock + threadIdx.x;
  int keep = 0;
  if (c < S.ncand) {
    float th = 0.0f;
    for (int q = 0; q < S.slices; ++q) th += S.theta[(int64_t)q * S.ncand + c];
    keep = th > 3.14159265358979324f;
    S.flag[c] = (uint8_t)keep;
  }
  const int cnt = __syncthreads_count(keep);
  if (threadIdx.x == 0) S.bcount[blockIdx.x] = cnt;
}

// Stable scatter of kept candidates; weight f(y) |box| (p = 1/|box| on the box).
template <int D>
__global__ void __launch_bounds__(kSrcBlock) k_src_scatter(const SrcParams S) {
  __shared__ int wsum[kSrcBlock / 32];
  const int64_t c = blockIdx.x * (int64_t)kSrcBlock + threadIdx.x;
  const int keep = c < S.ncand ? S.flag[c] : 0;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned bal = __ballot_sync(0xffffffffu, keep);
  if (lane == 0) wsum[w] = __popc(bal);
  __syncthreads();
  int before = 0;
  for (int q = 0; q < w; ++q) before += wsum[q];
  before += __popc(bal & ((1u << lane) - 1u));
  if (keep) {
    const int64_t j = S.boff[blockIdx.x] + before;
    float y[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      y[a] = S.yc[a * S.ncand + c];
      S.src_y[a * S.ncand + j] = y[a];
    }
    S.src_c[j] = (double)eval_fn<D>(S.f, y) * S.box;
  }
}

// dL/dA_k += sum_j dL/dc_j |box| psi_k(y_j) over the kept candidates (c_j =
// f(y_j) |box|): FP64 per thread, fixed-order warp sums, one atomic per warp.
template <int D>
__global__ void __launch_bounds__(256) k_src_adjoint(DevFunction f, const float* __restrict__ src_y, int64_t ncand,
                                                    const int64_t* __restrict__ n_src, double box,
                                                    const double* __restrict__ adj, double* __restrict__ grad_amp) {
  double acc[kMaxBumps];
#pragma unroll
  for (int b = 0; b < kMaxBumps; ++b) acc[b] = 0.0;
  const int64_t nk = *n_src;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nk; j += (int64_t)gridDim.x * blockDim.x) {
    float y[D];
#pragma unroll
    for (int a = 0; a < D; ++a) y[a] = src_y[a * ncand + j];
    float psi[kMaxBumps];
    bump_shapes<D>(f, y, psi);
    const double a = adj[j] * box;
#pragma unroll
    for (int b = 0; b < kMaxBumps; ++b) acc[b] += a * (double)psi[b];
  }
#pragma unroll
  for (int b = 0; b < kMaxBumps; ++b) {
    double v = acc[b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(&grad_amp[b], v);
  }
}

// Weights of already-kept candidates: c_j = f(y_j) |box| (as k_src_scatter).
template <int D>
__global__ void __launch_bounds__(256) k_src_reweight(DevFunction f, const float* __restrict__ src_y, int64_t ncand,
                                                     const int64_t* __restrict__ n_src, double box,
                                                     double* __restrict__ src_c) {
  const int64_t nk = *n_src;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nk; j += (int64_t)gridDim.x * blockDim.x) {
    float y[D];
#pragma unroll
    for (int a = 0; a < D; ++a) y[a] = src_y[a * ncand + j];
    src_c[j] = (double)eval_fn<D>(f, y) * box;
  }
}

}  // namespace bvc

using namespace bvc;

namespace bvc {
bvc_status bvc_source_reweight(bvc_geometry g, const bvc_function* ffn, bvc_cache* cache, cudaStream_t s) {
  DevFunction f;
  if (!make_dev_function(ffn, g->dim, &f)) return BVC_ERR_INVALID_ARG;
  double box = 1.0;
  for (int a = 0; a < g->dim; ++a) box *= (double)g->hi[a] - (double)g->lo[a];
  int64_t blocks = (cache->n_src_cand + 255) / 256;
  const int64_t cap = (int64_t)num_sms() * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  ProfScope ps("source_reweight", s);
  if (g->dim == 2)
    k_src_reweight<2><<<(unsigned)blocks, 256, 0, s>>>(f, cache->src_y, cache->n_src_cand, cache->n_src_dev, box,
                                                       cache->src_c);
  else
    k_src_reweight<3><<<(unsigned)blocks, 256, 0, s>>>(f, cache->src_y, cache->n_src_cand, cache->n_src_dev, box,
                                                       cache->src_c);
  BVC_LAUNCH_CHECK();
  return BVC_OK;
}

bvc_status bvc_source_adjoint(bvc_geometry g, const bvc_function* ffn, const bvc_cache* cache, const double* adj,
                              double* grad_amp, cudaStream_t s) {
  DevFunction f;
  if (!make_dev_function(ffn, g->dim, &f)) return BVC_ERR_INVALID_ARG;
  double box = 1.0;
  for (int a = 0; a < g->dim; ++a) box *= (double)g->hi[a] - (double)g->lo[a];
  int64_t blocks = (cache->n_src_cand + 255) / 256;
  const int64_t cap = (int64_t)num_sms() * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  ProfScope ps("adjoint_source", s);
  if (g->dim == 2)
    k_src_adjoint<2><<<(unsigned)blocks, 256, 0, s>>>(f, cache->src_y, cache->n_src_cand, cache->n_src_dev, box, adj,
                                                      grad_amp);
  else
    k_src_adjoint<3><<<(unsigned)blocks, 256, 0, s>>>(f, cache->src_y, cache->n_src_cand, cache->n_src_dev, box, adj,
                                                      grad_amp);
  BVC_LAUNCH_CHECK();
  return BVC_OK;
}
}  // namespace bvc

static size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

static bvc_status bvc_sample_source_workspace_size_impl(int64_t n_cand, size_t* bytes) {
  if (n_cand < 0 || bytes == nullptr) return BVC_ERR_INVALID_ARG;
  const int64_t nb = (n_cand + kSrcBlock - 1) / kSrcBlock;
  *bytes = al256((size_t)n_cand * 3 * sizeof(float)) + al256((size_t)n_cand) + 2 * al256((size_t)nb * 8) +
           al256((size_t)n_cand * kMaxSlices * sizeof(float));
  return BVC_OK;
}
extern "C" bvc_status bvc_sample_source_workspace_size(int64_t n_cand, size_t* bytes) {
  return bvc::note_status(bvc_sample_source_workspace_size_impl(n_cand, bytes));
}

static bvc_status bvc_sample_source_impl(bvc_geometry g, const bvc_function* ffn, const int32_t grid[3], uint64_t seed,
                                        double offset_l, bvc_cache* cache, void* workspace, size_t workspace_bytes,
                                        bvc_stream stream) {
  if (g == nullptr || grid == nullptr || cache == nullptr || !std::isfinite(offset_l) || offset_l < 0.0)
    return BVC_ERR_INVALID_ARG;
  const int D = g->dim;
  const int64_t ncand = (int64_t)grid[0] * grid[1] * (D == 3 ? grid[2] : 1);
  if (grid[0] < 1 || grid[1] < 1 || (D == 3 && grid[2] < 1) || ncand != cache->n_src_cand ||
      cache->src_y == nullptr || cache->src_c == nullptr || cache->n_src_dev == nullptr || workspace == nullptr)
    return BVC_ERR_INVALID_ARG;
  size_t need = 0;
  bvc_sample_source_workspace_size(ncand, &need);
  if (workspace_bytes < need) return BVC_ERR_WORKSPACE;
  SrcParams S{};
  S.G = g->dev;
  S.l = offset_l;
  if (!make_dev_function(ffn, D, &S.f)) return BVC_ERR_INVALID_ARG;
  S.G0 = grid[0];
  S.G1 = grid[1];
  S.G2 = D == 3 ? grid[2] : 1;
  S.seed = seed;
  S.lo0 = g->lo[0];
  S.lo1 = g->lo[1];
  S.lo2 = g->lo[2];
  const double ext0 = (double)g->hi[0] - (double)g->lo[0], ext1 = (double)g->hi[1] - (double)g->lo[1];
  const double ext2 = D == 3 ? (double)g->hi[2] - (double)g->lo[2] : 1.0;
  S.h0 = ext0 / grid[0];
  S.h1 = ext1 / grid[1];
  S.h2 = ext2 / S.G2;
  S.box = ext0 * ext1 * ext2;
  S.ncand = ncand;
  S.nblocks = (ncand + kSrcBlock - 1) / kSrcBlock;
  char* w = (char*)workspace;
  S.yc = (float*)w;
  w += al256((size_t)ncand * 3 * sizeof(float));
  S.flag = (uint8_t*)w;
  w += al256((size_t)ncand);
  S.bcount = (int64_t*)w;
  w += al256((size_t)S.nblocks * 8);
  S.boff = (int64_t*)w;
  w += al256((size_t)S.nblocks * 8);
  S.theta = (float*)w;
  if (D == 3) {  // about 8 blocks per SM, at least one tile of triangles per slice
    const int64_t want = ((int64_t)num_sms() * 8 + S.nblocks - 1) / S.nblocks;
    const int64_t tiles = (g->n_prims + kTriTile - 1) / kTriTile;
    S.slices = (int32_t)std::max<int64_t>(1, std::min<int64_t>({want, tiles, (int64_t)kMaxSlices}));
  }
  S.src_y = cache->src_y;
  S.src_c = cache->src_c;
  S.n_src = cache->n_src_dev;
  cudaStream_t s = (cudaStream_t)stream;
  {
    ProfScope ps("source_classify", s);
    if (D == 2) {
      k_src_classify<<<(unsigned)S.nblocks, kSrcBlock, 0, s>>>(S);
    } else {
      k_src_classify3d<<<dim3((unsigned)S.nblocks, (unsigned)S.slices), kSrcBlock, 0, s>>>(S);
      k_src_flag3d<<<(unsigned)S.nblocks, kSrcBlock, 0, s>>>(S);
    }
  }
  {
    ProfScope ps("source_scan", s);
    k_src_scan<<<1, 1024, 0, s>>>(S);
  }
  {
    ProfScope ps("source_scatter", s);
    if (D == 2)
      k_src_scatter<2><<<(unsigned)S.nblocks, kSrcBlock, 0, s>>>(S);
    else
      k_src_scatter<3><<<(unsigned)S.nblocks, kSrcBlock, 0, s>>>(S);
  }
  BVC_LAUNCH_CHECK();
  return BVC_OK;
}
extern "C" bvc_status bvc_sample_source(bvc_geometry g, const bvc_function* ffn, const int32_t grid[3], uint64_t seed,
                                        double offset_l, bvc_cache* cache, void* workspace, size_t workspace_bytes,
                                        bvc_stream stream) {
  return bvc::note_status(bvc_sample_source_impl(g, ffn, grid, seed, offset_l, cache, workspace, workspace_bytes, stream));
}
