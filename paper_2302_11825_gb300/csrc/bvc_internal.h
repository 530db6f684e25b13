// bvc_internal.h -- structures shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include <cstddef>
#include <cstdint>

#include "../../include/bvc.h"

namespace bvc {

__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }

// A problem function in device form, passed by value as a kernel parameter.
// Per term: kind, offset and count of its coefficients in c[] (FP32).
// GAUSS is stored as [-1/(2s^2), (A, centre)...]; GAUSS_LAPLACIAN as
// [-1/(2s^2), 1/s^4, -dim/s^2, (A, centre)...]; POLY and EXP_TRIG verbatim.
struct DevFunction {
  int32_t n_terms;
  int32_t kind[BVC_MAX_TERMS];
  int32_t off[BVC_MAX_TERMS];
  int32_t nc[BVC_MAX_TERMS];
  float c[BVC_MAX_COEFFS + 8];
};

// Device view of the geometry, passed by value to kernels.
//  nodes: 2D 3 float4 per node  [L.lo.x L.lo.y L.hi.x L.hi.y] [R ...] [cl cr - -]
//         3D 4 float4 per node  [L.lo.xyz L.hi.x] [L.hi.yz R.lo.xy] [R.lo.z R.hi.xyz] [cl cr - -]
//         child >= 0: internal node; child < 0: leaf, ~child = first << 4 | count.
//  slabs: per node, both children's slabs (unit normal n, dmin <= n.x <= dmax
//         over the elements below; n = 0 unbounded): 2D 2 float4
//         [n0 dmin0 dmax0] [n1 dmin1 dmax1]; 3D 3 float4
//         [n0 dmin0] [dmax0 n1] [dmin1 dmax1 - -] (see bvh_build.cpp).
//  prims: BVH order; 2D two float4 (a, ab) (1/|ab|^2, id, -, -); 3D three
//         float4 (a, id) (ab, -) (ac, -); id = caller's element index (int bits).
struct DevGeometry {
  const float4* nodes;
  const float4* slabs;
  const float4* prims;
  const double* cdf;      // [n_prims + 1] FP64 prefix sums of element measures (caller order)
  const float* verts;     // [n_verts][dim] caller's vertices
  const int32_t* idx;     // [n_prims][dim] caller's element indices
  const double* disp;     // [n_verts][dim] offset-boundary displacements m_v (Sec. 3.2)
  unsigned long long* stats;  // [4] status block
  int64_t n_prims, n_verts, n_nodes;
  float tau;              // traversal slack, 2^-18 x bbox diagonal
  float reach;            // max_v |m_v| (FP32, rounded up)
  float lo[3], hi[3];     // bbox
};

// One mesh of a batch (bvc_batch): its tree inside the forest, its shell,
// measure and its sample, point and gather-block ranges.
struct BatchMeshDev {
  int32_t root;     // forest node index of the mesh's root
  float eps;        // epsilon-shell
  double measure;   // |dOmega|
  int64_t smp_off, n_smp;
  int64_t pt_off, n_pts;
  int64_t blk_off;  // first gather block of the mesh (256 points per block)
};

constexpr int kStatSteps = 0, kStatCapped = 1, kStatFlags = 2, kStatCounter = 3, kStatNodes = 4, kStatPrims = 5;
constexpr unsigned long long kFlagTimeout = 1ull;
constexpr unsigned long long kFlagBounds = 2ull;  // a debug build's bounds check failed

}  // namespace bvc

struct bvc_batch_s {
  int32_t dim, count, walks, max_steps, k;
  int32_t counting;
  int64_t n_total, m_total, blocks_total;
  std::vector<bvc::BatchMeshDev> mesh;  // host copy of the table
  std::vector<double> offset_l;
  std::vector<bvc_geometry> geoms;      // borrowed
  void* arena;
  size_t arena_bytes;
  bvc::DevGeometry forest;              // concatenated nodes and primitives
  int32_t* sample_mesh;                 // [n_total] mesh of every sample
  bvc::BatchMeshDev* table;             // [count]
};

struct bvc_geometry_s {
  int32_t dim;
  int64_t n_verts, n_prims, n_nodes;
  double measure;
  double reach;           // max_v |m_v| of the offset boundary's displacements
  float lo[3], hi[3];
  void* arena;            // one device allocation holding everything below
  size_t arena_bytes;
  int32_t counting;       // walks count node fetches and primitive tests
  // Walk launch shape picked by bvc_tune_walks (0 = defaults): resident
  // blocks per SM of the persistent grid and walks per warp refill.
  int32_t tune_blocks_per_sm, tune_chunk;
  bvc::DevGeometry dev;
};

namespace bvc {

// Offset boundary (Sec. 3.2): per-vertex displacements m_v [n_verts][dim] of
// the closed surface v -> v - l m_v, from the unit normals of the elements
// at v that are moved (fixed[e] != 0: element e is not moved; may be NULL).
// 2D: k = 2 moved segments, S = na + nb: m = S / max(|S|^2 / 2, 1/4) (the
// miter); other k >= 1: S / |S|.  3D: angle-weighted normal N^, m = N^ /
// max(min_f n_f . N^, 1/4).  FP64 with a fixed operation order.  Returns
// max_v |m_v|.  (bvc_geometry.cu)
double offset_disp(int dim, const float* V, int64_t nv, const int32_t* F, int64_t np, const uint8_t* fixed,
                   double* m);

// The last status other than BVC_OK that an entry point returned on this
// thread (bvc_last_error); every extern "C" entry point passes its result
// through note_status.  (bvc_common.cu)
extern thread_local bvc_status g_last_status;
inline bvc_status note_status(bvc_status s) {
  if (s != BVC_OK) g_last_status = s;
  return s;
}

// Host helpers (bvc_common.cu)
bool make_dev_function(const bvc_function* f, int dim, DevFunction* out);
int num_sms();
// Pointwise walks (kRecGrad records) from the starts [i0, i0 + c) of a
// [dim][pt_stride] point set, walk ids wid0 + r * W + j, on geometry g; the
// records' U plane is then at walk_records_u(ws, c, dim)[r * W + j].
bvc_status walk_points_u(bvc_geometry g, const bvc_function* gfn, const bvc_function* ffn, double sigma,
                         const float* starts, int64_t pt_stride, int64_t i0, int64_t c, int32_t W, float eps,
                         int32_t max_steps, uint64_t seed, uint32_t tag, uint64_t wid0, void* ws, size_t ws_bytes,
                         cudaStream_t s);
const float* walk_records_u(void* ws, int64_t c, int dim);
// Weights f(y)|box| of the kept source samples already in the cache.
bvc_status bvc_source_reweight(bvc_geometry g, const bvc_function* ffn, bvc_cache* cache, cudaStream_t s);
// dL/dA of the source cache's bump amplitudes from dL/dc of its samples.
bvc_status bvc_source_adjoint(bvc_geometry g, const bvc_function* ffn, const bvc_cache* cache, const double* adj,
                              double* grad_amp, cudaStream_t s);
// seed_dev: when non-null, the seed is read from this device word at run
// time (a captured CUDA graph replays with the seed it holds then).
// zero_l: when non-null, samples on elements e with zero_l[e] != 0 keep
// offset 0 (the Neumann part of a mixed boundary).  disp: displacement table
// of the offset boundary (device double[n_verts][dim]); null = the
// geometry's own.  jac: device float[n] (plane of one float per sample).
bvc_status launch_sample_boundary(bvc_geometry g, int64_t n, double l, uint64_t seed, float* z, float* nrm,
                                  float* jac, int32_t* elem, int64_t stride, cudaStream_t s,
                                  const uint64_t* seed_dev, const uint8_t* zero_l = nullptr,
                                  const double* disp = nullptr);
// Per-start FP64 reduction of walk records (K3).
struct ReduceParams {
  const float* rec;
  int64_t n;       // starts in this launch
  int32_t W;
  int32_t planes;  // 1 + extra planes
  int64_t stride;  // plane stride of rec
  int32_t mode;    // 0 mean, 1 accumulate sum
  double* out[4];  // per plane, already offset to the launch's first start
};
bvc_status launch_reduce(const ReduceParams& R, cudaStream_t s);
int max_blocks_per_sm(const void* kernel, int block, size_t smem);

// Kernel timing: while bvc_profile_begin .. bvc_profile_end is active, every
// kernel launch of the library is bracketed by CUDA events recorded on the
// stream it is launched on.  ProfScope is placed around exactly one launch.
class ProfScope {
 public:
  ProfScope(const char* name, cudaStream_t s);
  ~ProfScope();
  ProfScope(const ProfScope&) = delete;
  ProfScope& operator=(const ProfScope&) = delete;

 private:
  int slot_;
  cudaStream_t s_;
};

}  // namespace bvc

#define BVC_CUDA_TRY(expr)                         \
  do {                                             \
    cudaError_t e_ = (expr);                       \
    if (e_ != cudaSuccess) return BVC_ERR_CUDA;    \
  } while (0)

#define BVC_LAUNCH_CHECK()                                   \
  do {                                                       \
    if (cudaPeekAtLastError() != cudaSuccess) {              \
      (void)cudaGetLastError();                              \
      return BVC_ERR_CUDA;                                   \
    }                                                        \
  } while (0)
