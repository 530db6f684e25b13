// bvc_gather.cu -- the all-pairs gather (K5, Eq. 3-6 / Alg. 1 splat loops),
// the cache packing that feeds it, and Alg. 1's GetSolution.
//
// Per pair the terms are FP32: 2D needs one reciprocal and one log2 of r^2
// (both on the SFU), 3D one reciprocal square root; everything else is FMA.
// Cache samples are packed with 1/p and the Green's-function constants of
// App. A folded into per-sample coefficients:
//   2D boundary (8 floats):  z.x z.y n.x n.y | a 2a b b ln2/2
//      a = u^ |dOmega| / (2 pi), b = du/dn^ |dOmega| / (2 pi)
//      u    += a (n.d)/r^2 - b ln r
//      grad += d (2a (n.d)/r^2 + b)/r^2 - a n / r^2            (d = z - x)
//   3D boundary (12 floats): z n a b 3a (a, b with 4 pi)
//      u    += a (n.d)/r^3 + b/r
//      grad += d (3a (n.d)/r^2 + b)/r^3 - a n / r^3
//   2D source (4 floats): y.x y.y c/(2 pi) c ln2/(4 pi):  u += c/(2 pi) ln r,  grad -= c/(2 pi) d/r^2
//   3D source (4 floats): y c/(4 pi):                    u -= c/(4 pi)/r,     grad -= c/(4 pi) d/r^3
// (G_2D = ln r/(2 pi), G_3D = -1/(4 pi r), the sign that makes Eq. 2 hold.)
//
// Tiles of 128 samples are brought into shared memory by bulk asynchronous
// copies (cp.async.bulk, completion on an mbarrier), double-buffered; one
// thread issues them while 256 threads each carry 4 evaluation points.  The
// FP32 sums over a tile are added to FP64 accumulators once per tile.
// Large cache sizes are split across CTAs; split partials are reduced in a
// fixed order, so results are deterministic.
#include <cmath>

#include "bvc_internal.h"

namespace bvc {

constexpr int kGBlock = 256;
constexpr int kGPts = 4;       // evaluation points per thread
constexpr int kTile = 128;     // samples per tile (FP32 partial-sum length)
constexpr int kPtsPerCta = kGBlock * kGPts;

__device__ unsigned long long g_gather_status = 0ull;

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_timer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait: gives up after ~2 s or 2^26 polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t phase) {
  if (mbar_try_wait(bar, phase)) return true;
  const uint64_t t0 = global_timer();
  for (int it = 0; it < (1 << 26); ++it) {
    if (mbar_try_wait(bar, phase)) return true;
    if ((it & 255) == 0 && global_timer() - t0 > 2000000000ull) break;
  }
  return false;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// ------------------------------------------------------------ pair terms
template <bool GRAD>
__device__ __forceinline__ void pair_bnd2(const float4 A, const float4 B, const float* p, float* acc) {
  const float dx = A.x - p[0], dy = A.y - p[1];
  const float r2 = fmaf(dy, dy, dx * dx);
  const float inv = rcp_approx(r2);
  const float l2 = lg2_approx(r2);
  const float nd = fmaf(A.w, dy, A.z * dx);
  const float s = nd * inv;
  acc[0] = fmaf(B.x, s, acc[0]);
  acc[0] = fmaf(-B.w, l2, acc[0]);
  if (GRAD) {
    const float ai = B.x * inv;
    const float k = fmaf(B.y, s, B.z) * inv;
    acc[1] = fmaf(k, dx, acc[1]);
    acc[1] = fmaf(-ai, A.z, acc[1]);
    acc[2] = fmaf(k, dy, acc[2]);
    acc[2] = fmaf(-ai, A.w, acc[2]);
  }
}

template <bool GRAD>
__device__ __forceinline__ void pair_bnd3(const float4 A, const float4 B, const float4 C, const float* p,
                                          float* acc) {
  const float dx = A.x - p[0], dy = A.y - p[1], dz = A.z - p[2];
  const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
  const float ir = rsqrt_approx(r2);
  const float ir2 = ir * ir;
  const float ir3 = ir2 * ir;
  const float nd = fmaf(B.z, dz, fmaf(B.y, dy, B.x * dx));
  acc[0] = fmaf(A.w * nd, ir3, acc[0]);
  acc[0] = fmaf(B.w, ir, acc[0]);
  if (GRAD) {
    const float k = fmaf(C.x, nd * ir2, B.w) * ir3;
    const float ai = A.w * ir3;
    acc[1] = fmaf(k, dx, acc[1]);
    acc[1] = fmaf(-ai, B.x, acc[1]);
    acc[2] = fmaf(k, dy, acc[2]);
    acc[2] = fmaf(-ai, B.y, acc[2]);
    acc[3] = fmaf(k, dz, acc[3]);
    acc[3] = fmaf(-ai, B.z, acc[3]);
  }
}

template <int D, bool GRAD>
__device__ __forceinline__ void pair_src(const float4 A, const float* p, float* acc) {
  if (D == 2) {
    const float dx = A.x - p[0], dy = A.y - p[1];
    const float r2 = fmaf(dy, dy, dx * dx);
    acc[0] = fmaf(A.w, lg2_approx(r2), acc[0]);
    if (GRAD) {
      const float ci = A.z * rcp_approx(r2);
      acc[1] = fmaf(-ci, dx, acc[1]);
      acc[2] = fmaf(-ci, dy, acc[2]);
    }
  } else {
    const float dx = A.x - p[0], dy = A.y - p[1], dz = A.z - p[2];
    const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    const float ir = rsqrt_approx(r2);
    acc[0] = fmaf(-A.w, ir, acc[0]);
    if (GRAD) {
      const float ci = A.w * ir * ir * ir;
      acc[1] = fmaf(-ci, dx, acc[1]);
      acc[2] = fmaf(-ci, dy, acc[2]);
      acc[3] = fmaf(-ci, dz, acc[3]);
    }
  }
}

// ------------------------------------------------------------ gather kernel
// KIND: 0 boundary, 1 source.  SPF: float4 per sample.
struct GatherArgs {
  const float* x;          // [D][m]
  int64_t m;
  const float4* samples;   // packed
  int64_t n;               // sample count (upper bound for sources)
  const int64_t* n_dev;    // device count (sources) or null
  int64_t split_len;       // samples per split (multiple of kTile)
  int32_t n_splits;
  int32_t pblocks;
  double* out[4];          // direct mode: running sums (u, grad a)
  double* part;            // split mode: [n_splits][planes][m]
};

template <int D, int KIND, bool GRAD>
__global__ void __launch_bounds__(kGBlock) k_gather(const GatherArgs A) {
  constexpr int SPF = KIND == 1 ? 1 : (D == 2 ? 2 : 3);
  constexpr int NA = GRAD ? 1 + D : 1;
  __shared__ __align__(128) float4 tile[2][kTile * SPF];
  __shared__ __align__(8) uint64_t bar[2];
  const int pb = blockIdx.x % A.pblocks;
  const int sp = blockIdx.x / A.pblocks;
  int64_t n = A.n;
  if (A.n_dev) n = min64(n, *A.n_dev);
  const int64_t s0 = (int64_t)sp * A.split_len;
  const int64_t s1 = min64(n, s0 + A.split_len);
  const int64_t nt = s1 > s0 ? (s1 - s0 + kTile - 1) / kTile : 0;

  // evaluation points of this thread (out-of-range points sit far away)
  float p[kGPts][D];
  int64_t kidx[kGPts];
#pragma unroll
  for (int j = 0; j < kGPts; ++j) {
    kidx[j] = (int64_t)pb * kPtsPerCta + j * kGBlock + threadIdx.x;
#pragma unroll
    for (int a = 0; a < D; ++a) p[j][a] = kidx[j] < A.m ? A.x[a * A.m + kidx[j]] : 1.0e4f + (float)a;
  }
  double acc64[kGPts][NA];
#pragma unroll
  for (int j = 0; j < kGPts; ++j)
#pragma unroll
    for (int q = 0; q < NA; ++q) acc64[j][q] = 0.0;

  if (nt > 0) {
    if (threadIdx.x == 0) {
      mbar_init(&bar[0], 1);
      mbar_init(&bar[1], 1);
      fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int b = 0; b < 2 && b < nt; ++b) {
        const int64_t st = s0 + (int64_t)b * kTile;
        const uint32_t cnt = (uint32_t)min64(kTile, s1 - st);
        mbar_expect_tx(&bar[b], cnt * SPF * 16u);
        bulk_g2s(&tile[b][0], A.samples + st * SPF, cnt * SPF * 16u, &bar[b]);
      }
    }
    for (int64_t it = 0; it < nt; ++it) {
      const int b = (int)(it & 1);
      const uint32_t phase = (uint32_t)((it >> 1) & 1);
      const bool ok = mbar_wait_bounded(&bar[b], phase);
      if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) atomicOr(&g_gather_status, 1ull);
        // give copies still in flight a bounded chance to land before exit
        if (threadIdx.x == 0)
          for (int64_t k2 = it; k2 < it + 2 && k2 < nt; ++k2)
            (void)mbar_wait_bounded(&bar[k2 & 1], (uint32_t)((k2 >> 1) & 1));
        return;
      }
      const int cnt = (int)min64(kTile, s1 - (s0 + it * kTile));
      float acc[kGPts][NA];
#pragma unroll
      for (int j = 0; j < kGPts; ++j)
#pragma unroll
        for (int q = 0; q < NA; ++q) acc[j][q] = 0.0f;
      const float4* T = tile[b];
#pragma unroll 2
      for (int s = 0; s < cnt; ++s) {
        if (KIND == 1) {
          const float4 S0 = T[s];
#pragma unroll
          for (int j = 0; j < kGPts; ++j) pair_src<D, GRAD>(S0, p[j], acc[j]);
        } else if (D == 2) {
          const float4 S0 = T[2 * s], S1 = T[2 * s + 1];
#pragma unroll
          for (int j = 0; j < kGPts; ++j) pair_bnd2<GRAD>(S0, S1, p[j], acc[j]);
        } else {
          const float4 S0 = T[3 * s], S1 = T[3 * s + 1], S2 = T[3 * s + 2];
#pragma unroll
          for (int j = 0; j < kGPts; ++j) pair_bnd3<GRAD>(S0, S1, S2, p[j], acc[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < kGPts; ++j)
#pragma unroll
        for (int q = 0; q < NA; ++q) acc64[j][q] += (double)acc[j][q];
      __syncthreads();  // every thread is done with tile[b]
      if (threadIdx.x == 0 && it + 2 < nt) {
        fence_proxy_async();
        const int64_t st = s0 + (it + 2) * kTile;
        const uint32_t c2 = (uint32_t)min64(kTile, s1 - st);
        mbar_expect_tx(&bar[b], c2 * SPF * 16u);
        bulk_g2s(&tile[b][0], A.samples + st * SPF, c2 * SPF * 16u, &bar[b]);
      }
    }
  }
  // results
#pragma unroll
  for (int j = 0; j < kGPts; ++j) {
    const int64_t k = kidx[j];
    if (k >= A.m) continue;
    if (A.n_splits == 1) {
      if (nt > 0)
#pragma unroll
        for (int q = 0; q < NA; ++q) A.out[q][k] += acc64[j][q];
    } else {
#pragma unroll
      for (int q = 0; q < NA; ++q) A.part[((int64_t)sp * NA + q) * A.m + k] = acc64[j][q];
    }
  }
}

// Fixed-order sum of split partials into the running sums.
__global__ void __launch_bounds__(256) k_gather_reduce(const GatherArgs A, int planes) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < A.m; k += (int64_t)gridDim.x * blockDim.x) {
    for (int q = 0; q < planes; ++q) {
      double s = 0.0;
      for (int sp = 0; sp < A.n_splits; ++sp) s += A.part[((int64_t)sp * planes + q) * A.m + k];
      A.out[q][k] += s;
    }
  }
}

__global__ void k_add_counts(int64_t* counts, int64_t nb, int64_t ns) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    counts[0] += nb;
    counts[1] += ns;
  }
}

// ------------------------------------------------------------ packing
template <int D>
__global__ void __launch_bounds__(256) k_pack_bnd(const bvc_cache C) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= C.n) return;
  const double two_pi = 6.283185307179586476925, four_pi = 12.566370614359172953850;
  if (D == 2) {
    const double a = C.u_hat[i] * C.bnd_measure / two_pi;
    const double b = C.dudn_hat[i] * C.bnd_measure / two_pi;
    float4* o = (float4*)C.packed + 2 * i;
    o[0] = make_float4(C.z[i], C.z[C.n + i], C.nrm[i], C.nrm[C.n + i]);
    o[1] = make_float4((float)a, (float)(2.0 * a), (float)b, (float)(b * 0.34657359027997265471));
  } else {
    const double a = C.u_hat[i] * C.bnd_measure / four_pi;
    const double b = C.dudn_hat[i] * C.bnd_measure / four_pi;
    float4* o = (float4*)C.packed + 3 * i;
    o[0] = make_float4(C.z[i], C.z[C.n + i], C.z[2 * C.n + i], (float)a);
    o[1] = make_float4(C.nrm[i], C.nrm[C.n + i], C.nrm[2 * C.n + i], (float)b);
    o[2] = make_float4((float)(3.0 * a), 0.0f, 0.0f, 0.0f);
  }
}

template <int D>
__global__ void __launch_bounds__(256) k_pack_src(const bvc_cache C) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= C.n_src_cand || j >= *C.n_src_dev) return;
  const double c = C.src_c[j];
  float4* o = (float4*)C.src_packed + j;
  const int64_t M = C.n_src_cand;
  if (D == 2) {
    const double c1 = c / 6.283185307179586476925;
    o[0] = make_float4(C.src_y[j], C.src_y[M + j], (float)c1, (float)(c1 * 0.34657359027997265471));
  } else {
    o[0] = make_float4(C.src_y[j], C.src_y[M + j], C.src_y[2 * M + j], (float)(c / 12.566370614359172953850));
  }
}

template <int D>
__global__ void __launch_bounds__(256) k_get_solution(const bvc_eval_state S, double* u, double* grad) {
  const int64_t nb = S.counts[0], ns = S.counts[1];
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < S.m; k += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    if (nb > 0) v += S.u_bnd[k] / (double)nb;
    if (ns > 0) v += S.u_src[k] / (double)ns;
    u[k] = v;
    if (grad)
      for (int a = 0; a < D; ++a) {
        double gv = 0.0;
        if (nb > 0 && S.grad_bnd) gv += S.grad_bnd[a * S.m + k] / (double)nb;
        if (ns > 0 && S.grad_src) gv += S.grad_src[a * S.m + k] / (double)ns;
        grad[a * S.m + k] = gv;
      }
  }
}

struct Plan {
  int32_t pblocks, n_splits;
  int64_t split_len;
};

static Plan plan_gather(int64_t m, int64_t n, const void* kern) {
  Plan P;
  P.pblocks = (int32_t)((m + kPtsPerCta - 1) / kPtsPerCta);
  const int64_t tiles = (n + kTile - 1) / kTile;
  const int64_t conc = (int64_t)num_sms() * max_blocks_per_sm(kern, kGBlock, 0);
  int64_t want = (4 * conc + P.pblocks - 1) / P.pblocks;
  if (want > 16) want = 16;
  if (want > tiles) want = tiles;
  if (want < 1) want = 1;
  const int64_t tiles_per = (tiles + want - 1) / want;
  P.split_len = (tiles_per > 0 ? tiles_per : 1) * kTile;
  P.n_splits = (int32_t)((n + P.split_len - 1) / P.split_len);
  if (P.n_splits < 1) P.n_splits = 1;
  return P;
}

template <int D, int KIND, bool GRAD>
static const void* gather_kernel() {
  return (const void*)k_gather<D, KIND, GRAD>;
}

static const void* pick(int D, int kind, bool grad) {
  if (D == 2) {
    if (kind == 0) return grad ? gather_kernel<2, 0, true>() : gather_kernel<2, 0, false>();
    return grad ? gather_kernel<2, 1, true>() : gather_kernel<2, 1, false>();
  }
  if (kind == 0) return grad ? gather_kernel<3, 0, true>() : gather_kernel<3, 0, false>();
  return grad ? gather_kernel<3, 1, true>() : gather_kernel<3, 1, false>();
}

static size_t part_bytes(const Plan& P, int planes, int64_t m) {
  return P.n_splits > 1 ? (size_t)P.n_splits * planes * (size_t)m * sizeof(double) : 0;
}

}  // namespace bvc

using namespace bvc;

extern "C" bvc_status bvc_cache_pack(const bvc_cache* cache, bvc_stream stream) {
  if (cache == nullptr || (cache->dim != 2 && cache->dim != 3) || cache->n < 0) return BVC_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (cache->n > 0) {
    if (!cache->z || !cache->nrm || !cache->u_hat || !cache->dudn_hat || !cache->packed) return BVC_ERR_INVALID_ARG;
    const unsigned grid = (unsigned)((cache->n + 255) / 256);
    ProfScope ps("pack_boundary", s);
    if (cache->dim == 2)
      k_pack_bnd<2><<<grid, 256, 0, s>>>(*cache);
    else
      k_pack_bnd<3><<<grid, 256, 0, s>>>(*cache);
  }
  if (cache->n_src_cand > 0) {
    if (!cache->src_y || !cache->src_c || !cache->src_packed || !cache->n_src_dev) return BVC_ERR_INVALID_ARG;
    const unsigned grid = (unsigned)((cache->n_src_cand + 255) / 256);
    ProfScope ps("pack_source", s);
    if (cache->dim == 2)
      k_pack_src<2><<<grid, 256, 0, s>>>(*cache);
    else
      k_pack_src<3><<<grid, 256, 0, s>>>(*cache);
  }
  BVC_LAUNCH_CHECK();
  return BVC_OK;
}

extern "C" bvc_status bvc_evaluate_workspace_size(const bvc_cache* cache, const bvc_eval_state* state,
                                                  size_t* bytes) {
  if (cache == nullptr || state == nullptr || bytes == nullptr || cache->dim != state->dim) return BVC_ERR_INVALID_ARG;
  const int D = cache->dim;
  const bool grad = state->grad_bnd != nullptr;
  const int planes = grad ? 1 + D : 1;
  size_t b = 0;
  if (cache->n > 0) {
    const Plan P = plan_gather(state->m, cache->n, pick(D, 0, grad));
    b = part_bytes(P, planes, state->m);
  }
  if (cache->n_src_cand > 0) {
    const Plan P = plan_gather(state->m, cache->n_src_cand, pick(D, 1, grad));
    const size_t bs = part_bytes(P, planes, state->m);
    b = bs > b ? bs : b;
  }
  *bytes = b;
  return BVC_OK;
}

static bvc_status run_part(int D, int kind, bool grad, const float* x, int64_t m, const float4* samples, int64_t n,
                           const int64_t* n_dev, double* u, double* g, void* ws, size_t ws_bytes, cudaStream_t s) {
  const void* kern = pick(D, kind, grad);
  const Plan P = plan_gather(m, n, kern);
  const int planes = grad ? 1 + D : 1;
  GatherArgs A{};
  A.x = x;
  A.m = m;
  A.samples = samples;
  A.n = n;
  A.n_dev = n_dev;
  A.split_len = P.split_len;
  A.n_splits = P.n_splits;
  A.pblocks = P.pblocks;
  A.out[0] = u;
  for (int a = 0; a < D && grad; ++a) A.out[1 + a] = g + (int64_t)a * m;
  if (P.n_splits > 1) {
    if (ws == nullptr || ws_bytes < part_bytes(P, planes, m)) return BVC_ERR_WORKSPACE;
    A.part = (double*)ws;
  }
  void* args[] = {(void*)&A};
  {
    ProfScope ps(kind == 0 ? "gather_boundary" : "gather_source", s);
    BVC_CUDA_TRY(cudaLaunchKernel(kern, dim3((unsigned)(P.pblocks * P.n_splits)), dim3(kGBlock), args, 0, s));
  }
  if (P.n_splits > 1) {
    int64_t blocks = (m + 255) / 256;
    const int64_t cap = (int64_t)num_sms() * 8;
    if (blocks > cap) blocks = cap;
    ProfScope ps("gather_reduce", s);
    k_gather_reduce<<<(unsigned)blocks, 256, 0, s>>>(A, planes);
    BVC_LAUNCH_CHECK();
  }
  return BVC_OK;
}

extern "C" bvc_status bvc_evaluate(const bvc_cache* cache, bvc_eval_state* state, void* workspace,
                                   size_t workspace_bytes, bvc_stream stream) {
  if (cache == nullptr || state == nullptr || cache->dim != state->dim || (cache->dim != 2 && cache->dim != 3) ||
      state->m < 0 || cache->n < 0 || state->counts == nullptr)
    return BVC_ERR_INVALID_ARG;
  const int D = cache->dim;
  const bool grad = state->grad_bnd != nullptr;
  if (grad != (state->grad_src != nullptr)) return BVC_ERR_INVALID_ARG;
  if (state->m > 0 && (state->x == nullptr || state->u_bnd == nullptr || state->u_src == nullptr))
    return BVC_ERR_INVALID_ARG;
  if ((cache->n > 0 && cache->packed == nullptr) ||
      (cache->n_src_cand > 0 && (cache->src_packed == nullptr || cache->n_src_dev == nullptr)))
    return BVC_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (state->m > 0) {
    if (cache->n > 0) {
      bvc_status st = run_part(D, 0, grad, state->x, state->m, (const float4*)cache->packed, cache->n, nullptr,
                               state->u_bnd, state->grad_bnd, workspace, workspace_bytes, s);
      if (st != BVC_OK) return st;
    }
    if (cache->n_src_cand > 0) {
      bvc_status st = run_part(D, 1, grad, state->x, state->m, (const float4*)cache->src_packed, cache->n_src_cand,
                               cache->n_src_dev, state->u_src, state->grad_src, workspace, workspace_bytes, s);
      if (st != BVC_OK) return st;
    }
  }
  {
    ProfScope ps("add_counts", s);
    k_add_counts<<<1, 32, 0, s>>>(state->counts, cache->n, cache->n_src_cand);
  }
  BVC_LAUNCH_CHECK();
  return BVC_OK;
}

extern "C" bvc_status bvc_eval_state_reset(const bvc_eval_state* state, bvc_stream stream) {
  if (state == nullptr || state->m < 0 || state->counts == nullptr || (state->dim != 2 && state->dim != 3))
    return BVC_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t mb = (size_t)state->m * sizeof(double);
  if (state->m > 0) {
    if (state->u_bnd == nullptr || state->u_src == nullptr) return BVC_ERR_INVALID_ARG;
    BVC_CUDA_TRY(cudaMemsetAsync(state->u_bnd, 0, mb, s));
    BVC_CUDA_TRY(cudaMemsetAsync(state->u_src, 0, mb, s));
    if (state->grad_bnd) BVC_CUDA_TRY(cudaMemsetAsync(state->grad_bnd, 0, mb * state->dim, s));
    if (state->grad_src) BVC_CUDA_TRY(cudaMemsetAsync(state->grad_src, 0, mb * state->dim, s));
  }
  BVC_CUDA_TRY(cudaMemsetAsync(state->counts, 0, 2 * sizeof(int64_t), s));
  return BVC_OK;
}

extern "C" bvc_status bvc_get_solution(const bvc_eval_state* state, double* u, double* grad, bvc_stream stream) {
  if (state == nullptr || u == nullptr || state->m < 0 || state->counts == nullptr ||
      (state->dim != 2 && state->dim != 3))
    return BVC_ERR_INVALID_ARG;
  if (state->m == 0) return BVC_OK;
  int64_t blocks = (state->m + 255) / 256;
  const int64_t cap = (int64_t)num_sms() * 8;
  if (blocks > cap) blocks = cap;
  ProfScope ps("get_solution", (cudaStream_t)stream);
  if (state->dim == 2)
    k_get_solution<2><<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(*state, u, grad);
  else
    k_get_solution<3><<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(*state, u, grad);
  BVC_LAUNCH_CHECK();
  return BVC_OK;
}

extern "C" bvc_status bvc_gather_status(uint64_t* flags, int32_t reset) {
  if (flags == nullptr) return BVC_ERR_INVALID_ARG;
  unsigned long long h = 0;
  BVC_CUDA_TRY(cudaMemcpyFromSymbol(&h, g_gather_status, sizeof(h)));
  if (reset) {
    const unsigned long long z = 0;
    BVC_CUDA_TRY(cudaMemcpyToSymbol(g_gather_status, &z, sizeof(z)));
  }
  *flags = h;
  return (h & 1ull) ? BVC_ERR_TIMEOUT : BVC_OK;
}
