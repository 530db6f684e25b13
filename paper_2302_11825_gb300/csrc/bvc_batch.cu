// bvc_batch.cu -- batches of meshes: one BVH forest for independent
// problems on meshes of uneven size.
//
// The meshes' node and primitive arrays are copied into one device arena,
// mesh after mesh.  Child links of internal nodes move by the mesh's node
// offset and the first-primitive field of leaves by its primitive offset;
// element ids inside the primitive records stay mesh-local (they only break
// ties within one mesh).  The root of mesh j is its node offset.  A walk
// started at a sample of mesh j traverses only mesh j's tree, so its
// closest-point answers -- the canonical minimum over that mesh with ties to
// the lowest id -- are those of the mesh's own BVH: the forest's traversal
// slack (the largest over the meshes) can only add node visits.
#include <algorithm>
#include <cmath>

#include "bvc_internal.h"

namespace bvc {

// Copies n nodes, moving child links: internal children by node_off, leaf
// first-primitive fields by prim_off (leaf = ~(first << 4 | count)).
template <int D>
__global__ void __launch_bounds__(256) k_rebase_nodes(const float4* __restrict__ src, int64_t n,
                                                      float4* __restrict__ dst, int32_t node_off, int32_t prim_off) {
  constexpr int PER = D == 2 ? 3 : 4;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
#pragma unroll
  for (int a = 0; a < PER - 1; ++a) dst[PER * i + a] = src[PER * i + a];
  float4 c = src[PER * i + PER - 1];
  int32_t ch[2] = {__float_as_int(c.x), __float_as_int(c.y)};
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    if (ch[b] >= 0) {
      ch[b] += node_off;
    } else {
      const int32_t e = ~ch[b];
      ch[b] = ~((((e >> 4) + prim_off) << 4) | (e & 15));
    }
  }
  c.x = __int_as_float(ch[0]);
  c.y = __int_as_float(ch[1]);
  dst[PER * i + PER - 1] = c;
}

static size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace bvc

using namespace bvc;

static bvc_status bvc_batch_create_impl(const bvc_batch_mesh* meshes, int32_t count, int32_t walks, int32_t max_steps,
                                       int32_t k, bvc_stream stream, bvc_batch* out) {
  if (out == nullptr) return BVC_ERR_INVALID_ARG;
  *out = nullptr;
  if (meshes == nullptr || count < 1 || walks < 1 || max_steps < 1 || k < 1 || meshes[0].geom == nullptr)
    return BVC_ERR_INVALID_ARG;
  const int dim = meshes[0].geom->dim;
  int64_t n_nodes = 0, n_prims = 0, n_total = 0, m_total = 0, blocks = 0;
  float tau = 0.0f;
  std::vector<BatchMeshDev> tab(count);
  std::vector<double> offl(count);
  std::vector<bvc_geometry> geoms(count);
  for (int j = 0; j < count; ++j) {
    const bvc_batch_mesh& m = meshes[j];
    if (m.geom == nullptr || m.geom->dim != dim || m.n_samples < 1 || m.n_points < 0 || !std::isfinite(m.eps) ||
        !(m.eps > 0.0f) || !std::isfinite(m.offset_l) || !(m.offset_l > 0.0))
      return BVC_ERR_INVALID_ARG;
    BatchMeshDev& t = tab[j];
    t.root = (int32_t)n_nodes;
    t.eps = m.eps;
    t.measure = m.geom->measure;
    t.smp_off = n_total;
    t.n_smp = m.n_samples;
    t.pt_off = m_total;
    t.n_pts = m.n_points;
    t.blk_off = blocks;
    offl[j] = m.offset_l;
    geoms[j] = m.geom;
    n_nodes += m.geom->n_nodes;
    n_prims += m.geom->n_prims;
    n_total += m.n_samples;
    m_total += m.n_points;
    blocks += (m.n_points + 255) / 256;
    tau = std::max(tau, m.geom->dev.tau);
  }
  // leaf fields hold 27-bit primitive indices; node links are int32
  if (n_prims >= (int64_t(1) << 27) || n_nodes >= (int64_t(1) << 31)) return BVC_ERR_UNSUPPORTED;
  const int per_node = dim == 2 ? 3 : 4, per_prim = dim == 2 ? 2 : 3;
  const size_t b_nodes = align256((size_t)n_nodes * per_node * sizeof(float4));
  const int per_slab = dim == 2 ? 2 : 3;
  const size_t b_slabs = align256((size_t)n_nodes * per_slab * sizeof(float4));
  const size_t b_prims = align256((size_t)n_prims * per_prim * sizeof(float4));
  const size_t b_stats = 256;
  const size_t b_mesh = align256((size_t)n_total * sizeof(int32_t));
  const size_t b_tab = align256((size_t)count * sizeof(BatchMeshDev));
  bvc_batch b = new bvc_batch_s();
  b->dim = dim;
  b->count = count;
  b->walks = walks;
  b->max_steps = max_steps;
  b->k = k;
  b->n_total = n_total;
  b->m_total = m_total;
  b->blocks_total = blocks;
  b->mesh = tab;
  b->offset_l = offl;
  b->geoms = geoms;
  b->arena_bytes = b_nodes + b_slabs + b_prims + b_stats + b_mesh + b_tab;
  // stream-ordered, like bvc_geometry_create: ready for work on `stream`
  if (cudaMallocAsync(&b->arena, b->arena_bytes, (cudaStream_t)stream) != cudaSuccess) {
    (void)cudaGetLastError();
    delete b;
    return BVC_ERR_OOM;
  }
  char* base = (char*)b->arena;
  DevGeometry& F = b->forest;
  F = DevGeometry{};
  F.nodes = (const float4*)base;
  F.slabs = (const float4*)(base += b_nodes);
  F.prims = (const float4*)(base += b_slabs);
  F.stats = (unsigned long long*)(base += b_prims);
  b->sample_mesh = (int32_t*)(base += b_stats);
  b->table = (BatchMeshDev*)(base += b_mesh);
  F.n_prims = n_prims;
  F.n_nodes = n_nodes;
  F.tau = tau;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<int32_t> smesh((size_t)n_total);
  for (int j = 0; j < count; ++j)
    std::fill(smesh.begin() + tab[j].smp_off, smesh.begin() + tab[j].smp_off + tab[j].n_smp, j);
  bool ok = cudaMemsetAsync(F.stats, 0, b_stats, s) == cudaSuccess &&
            cudaMemcpyAsync(b->sample_mesh, smesh.data(), smesh.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                            s) == cudaSuccess &&
            cudaMemcpyAsync(b->table, tab.data(), tab.size() * sizeof(BatchMeshDev), cudaMemcpyHostToDevice, s) ==
                cudaSuccess;
  int64_t prim_off = 0;
  for (int j = 0; j < count && ok; ++j) {
    const bvc_geometry g = geoms[j];
    const int64_t nn = g->n_nodes;
    float4* dn = (float4*)F.nodes + (size_t)tab[j].root * per_node;
    if (dim == 2)
      k_rebase_nodes<2><<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(g->dev.nodes, nn, dn, tab[j].root,
                                                                      (int32_t)prim_off);
    else
      k_rebase_nodes<3><<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(g->dev.nodes, nn, dn, tab[j].root,
                                                                      (int32_t)prim_off);
    // slabs hold no links: copied as they are, node for node
    ok = cudaGetLastError() == cudaSuccess &&
         cudaMemcpyAsync((float4*)F.slabs + (size_t)tab[j].root * per_slab, g->dev.slabs,
                         (size_t)nn * per_slab * sizeof(float4), cudaMemcpyDeviceToDevice, s) == cudaSuccess &&
         cudaMemcpyAsync((float4*)F.prims + (size_t)prim_off * per_prim, g->dev.prims,
                         (size_t)g->n_prims * per_prim * sizeof(float4), cudaMemcpyDeviceToDevice, s) == cudaSuccess;
    prim_off += g->n_prims;
  }
  if (!ok) {
    (void)cudaGetLastError();
    (void)cudaFreeAsync(b->arena, s);
    delete b;
    return BVC_ERR_CUDA;
  }
  *out = b;
  return BVC_OK;
}
extern "C" bvc_status bvc_batch_create(const bvc_batch_mesh* meshes, int32_t count, int32_t walks, int32_t max_steps,
                                       int32_t k, bvc_stream stream, bvc_batch* out) {
  return bvc::note_status(bvc_batch_create_impl(meshes, count, walks, max_steps, k, stream, out));
}

static bvc_status bvc_batch_destroy_impl(bvc_batch b) {
  if (b == nullptr) return BVC_ERR_INVALID_ARG;
  const cudaError_t e = cudaFree(b->arena);
  delete b;
  return e == cudaSuccess ? BVC_OK : BVC_ERR_CUDA;
}
extern "C" bvc_status bvc_batch_destroy(bvc_batch b) {
  return bvc::note_status(bvc_batch_destroy_impl(b));
}

static bvc_status bvc_batch_set_counting_impl(bvc_batch b, int32_t on) {
  if (b == nullptr) return BVC_ERR_INVALID_ARG;
  b->counting = on ? 1 : 0;
  return BVC_OK;
}
extern "C" bvc_status bvc_batch_set_counting(bvc_batch b, int32_t on) {
  return bvc::note_status(bvc_batch_set_counting_impl(b, on));
}

static bvc_status bvc_batch_stats_impl(bvc_batch b, uint64_t out[8], int32_t reset, bvc_stream stream) {
  if (b == nullptr || out == nullptr) return BVC_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long h[8];
  BVC_CUDA_TRY(cudaMemcpyAsync(h, b->forest.stats, sizeof(h), cudaMemcpyDeviceToHost, s));
  if (reset) BVC_CUDA_TRY(cudaMemsetAsync(b->forest.stats, 0, sizeof(h), s));
  BVC_CUDA_TRY(cudaStreamSynchronize(s));
  for (int i = 0; i < 8; ++i) out[i] = h[i];
  if (h[kStatFlags] & kFlagBounds) return BVC_ERR_BOUNDS;
  if (h[kStatFlags] & kFlagTimeout) return BVC_ERR_TIMEOUT;
  if (h[kStatCapped]) return BVC_WARN_WALK_CAP;
  return BVC_OK;
}
extern "C" bvc_status bvc_batch_stats(bvc_batch b, uint64_t out[8], int32_t reset, bvc_stream stream) {
  return bvc::note_status(bvc_batch_stats_impl(b, out, reset, stream));
}

static bvc_status bvc_batch_get_info_impl(bvc_batch b, int32_t* dim, int64_t* n_total, int64_t* m_total) {
  if (b == nullptr) return BVC_ERR_INVALID_ARG;
  if (dim) *dim = b->dim;
  if (n_total) *n_total = b->n_total;
  if (m_total) *m_total = b->m_total;
  return BVC_OK;
}
extern "C" bvc_status bvc_batch_get_info(bvc_batch b, int32_t* dim, int64_t* n_total, int64_t* m_total) {
  return bvc::note_status(bvc_batch_get_info_impl(b, dim, n_total, m_total));
}
