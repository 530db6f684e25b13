// bvc_gather.cu -- the all-pairs gather (K5, Eq. 3-6 / Alg. 1 splat loops),
// the cache packing that feeds it, and Alg. 1's GetSolution.
//
// Per pair the terms are FP32: 2D needs one reciprocal and one log2 of r^2
// (both on the SFU), 3D one reciprocal square root; everything else is
// packed FP32x2 arithmetic (fma/mul/add .f32x2), two evaluation points per
// instruction.  Cache samples are packed with 1/p and the Green's-function
// constants of App. A folded into per-sample coefficients, each value
// stored twice so that one 16-byte shared-memory load yields two ready
// (value, value) operand pairs:
//   2D boundary (20 floats): z, n, a, -a, 2a, b, -b ln2/2
//      a = u^ |dOmega| / (2 pi), b = du/dn^ |dOmega| / (2 pi)
//      u    += a (n.d)/r^2 - b ln r
//      grad += d (2a (n.d)/r^2 + b)/r^2 - a n / r^2            (d = z - x)
//   3D boundary (20 floats): z, A = a n, -A, b   (a, b with 4 pi)
//      u    += (A.d)/r^3 + b/r
//      grad += (d (3 (A.d)/r^2 + b) - A) / r^3
//      (1/r from rsqrt and 1/r^2 from rcp, both on the SFU, so that the
//      FMA pipe carries 20 paired instructions per two pairs)
//   2D source (8 floats): y, c ln2/(4 pi), -c/(2 pi):  u += c/(2 pi) ln r,  grad -= c/(2 pi) d/r^2
//   3D source (8 floats): y, -c/(4 pi):                u -= c/(4 pi)/r,     grad -= c/(4 pi) d/r^3
// (G_2D = ln r/(2 pi), G_3D = -1/(4 pi r), the sign that makes Eq. 2 hold.)
//
// Tiles of 128 samples are brought into shared memory by bulk asynchronous
// copies (cp.async.bulk, completion on an mbarrier), double-buffered; one
// thread issues them while 256 threads each carry 6 (boundary) or 2
// (source) evaluation points.  The
// FP32 sums over a tile are added to FP64 accumulators once per tile
// (registers at 2 points per thread; shared memory, one slot per thread,
// point and plane, at 4 and 6, which frees the registers the wider shapes
// need: on GB300 the 6-point boundary gather went from 234 to 212 ms on
// the 1.31M-triangle sphere, ahead of the 2-point shape's 224 ms).
// Large cache sizes are split across CTAs; split partials are reduced in a
// fixed order, so results are deterministic.
#include <cmath>

#include "bvc_device.cuh"
#include "bvc_internal.h"

namespace bvc {

constexpr int kGBlock = 256;
// Tiles of 128 samples: FP32 partial sums over at most 128 samples keep the
// worst-case rounding below 128 x 2^-24 = 7.6e-6 of the sum of |terms|, inside
// the gather's 1e-5 tolerance.  (256-sample tiles, or flushing every 2 or 4
// tiles, were 1-4% faster on GB300 but double that worst case.)
#ifndef BVC_GATHER_TILE
#define BVC_GATHER_TILE 128
#endif
#ifndef BVC_GATHER_FLUSH
#define BVC_GATHER_FLUSH 1
#endif
// Samples per unrolled body of the pair loop (measured on GB300 with the
// autotuned shapes: 3D 2 / 4 / 8 -> 212.3 / 209.4 / 212.8 ms on the
// 1.31M-triangle sphere; 2D 2 / 4 / 8 -> 27.3 / 26.2 / 25.6 ms for the
// 20k-segment star's boundary and source gathers).
#ifndef BVC_GATHER_UNROLL_2D
#define BVC_GATHER_UNROLL_2D 8
#endif
#ifndef BVC_GATHER_UNROLL_3D
#define BVC_GATHER_UNROLL_3D 4
#endif
constexpr int kUnroll2 = BVC_GATHER_UNROLL_2D, kUnroll3 = BVC_GATHER_UNROLL_3D;
constexpr int kTile = BVC_GATHER_TILE;    // samples per tile copy
constexpr int kFlush = BVC_GATHER_FLUSH;  // tiles per FP32 partial sum (then added in FP64)
// Evaluation points per thread and resident CTAs per SM, per kind of sample
// (measured on GB300: boundary tiles are FMA/SFU-bound and gain from reuse
// of each shared-memory sample across 6 points; source tiles are SFU-bound
// and gain from occupancy).
// PTS evaluation points per thread: each sample loaded from shared memory
// serves PTS points; more points mean fewer loads per pair but more
// registers.  The supported counts are 2, 4, 6 (boundary) and 2, 4
// (source); the defaults below are the GB300 measurements' best, and
// bvc_tune_gather picks per workload.
template <int PTS>
struct GatherShape {
  static constexpr int kPts = PTS;
  static constexpr int kMinBlocks = PTS <= 2 ? 4 : (PTS == 4 ? 3 : 2);
  // FP64 per-point sums in shared memory (one slot per thread, point and
  // plane) instead of registers: frees 4 registers per sum for the wider
  // shapes, which only touch them once per tile
  static constexpr bool kSmemAcc = PTS >= 4;
  static constexpr int kPtsPerCta = kGBlock * PTS;
};
constexpr int kDefaultPts[2][2] = {{6, 2}, {4, 2}};  // [dim - 2][kind]
// the tuned counts (0 = default), process-wide: [dim - 2][kind]
static int g_gather_pts[2][2] = {{0, 0}, {0, 0}};
static int gather_pts(int D, int kind) {
  const int p = __atomic_load_n(&g_gather_pts[D - 2][kind], __ATOMIC_RELAXED);
  return p > 0 ? p : kDefaultPts[D - 2][kind];
}

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
// Bounded wait: gives up after limit_ns or 2^26 polls.
__device__ __forceinline__ bool mbar_wait_bounded_ns(uint64_t* bar, uint32_t phase, uint64_t limit_ns) {
  if (mbar_try_wait(bar, phase)) return true;
  const uint64_t t0 = global_timer();
  for (int it = 0; it < (1 << 26); ++it) {
    if (mbar_try_wait(bar, phase)) return true;
    if ((it & 255) == 0 && global_timer() - t0 > limit_ns) break;
  }
  return false;
}
// The gathers' wait for a tile copy: ~2 s.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t phase) {
  return mbar_wait_bounded_ns(bar, phase, 2000000000ull);
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

// ------------------------------------------------------------ packed FP32x2
typedef unsigned long long f2;  // two FP32 lanes in one 64-bit register pair
__device__ __forceinline__ f2 pk(float a, float b) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void upk(f2 v, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
  f2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
  f2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
  f2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 rcp2(f2 v) {
  float a, b;
  upk(v, a, b);
  return pk(rcp_approx(a), rcp_approx(b));
}
__device__ __forceinline__ f2 lg22(f2 v) {
  float a, b;
  upk(v, a, b);
  return pk(lg2_approx(a), lg2_approx(b));
}
__device__ __forceinline__ f2 rsqrt2(f2 v) {
  float a, b;
  upk(v, a, b);
  return pk(rsqrt_approx(a), rsqrt_approx(b));
}

// ------------------------------------------------------------ pair terms
// T: the sample's packed float4s viewed as pairs; (px, py[, pz]) hold -x of
// two evaluation points; acc = [u, grad...] pairs of the two points.
template <bool GRAD>
__device__ __forceinline__ void pair_bnd2(const ulonglong2* T, f2 px, f2 py, f2* acc) {
  const ulonglong2 zz = T[0], nn = T[1], aa = T[2], bb = T[3], cc = T[4];
  // zz = (z.x, z.y), nn = (n.x, n.y), aa = (a, -a), bb = (2a, b), cc = (-b ln2/2, -)
  const f2 dx = add2(zz.x, px), dy = add2(zz.y, py);
  const f2 r2 = fma2(dy, dy, mul2(dx, dx));
  const f2 inv = rcp2(r2);
  const f2 l2 = lg22(r2);
  const f2 nd = fma2(nn.y, dy, mul2(nn.x, dx));
  const f2 s = mul2(nd, inv);
  acc[0] = fma2(aa.x, s, acc[0]);
  acc[0] = fma2(cc.x, l2, acc[0]);
  if (GRAD) {
    const f2 nai = mul2(aa.y, inv);
    const f2 k = mul2(fma2(bb.x, s, bb.y), inv);
    acc[1] = fma2(nai, nn.x, fma2(k, dx, acc[1]));
    acc[2] = fma2(nai, nn.y, fma2(k, dy, acc[2]));
  }
}

template <bool GRAD>
__device__ __forceinline__ void pair_bnd3(const ulonglong2* T, f2 px, f2 py, f2 pz, f2* acc) {
  const ulonglong2 t0 = T[0], t1 = T[1], t2 = T[2], t3 = T[3], t4 = T[4];
  // t0 = (z.x, z.y), t1 = (z.z, A.x), t2 = (A.y, A.z), t3 = (-A.x, -A.y), t4 = (-A.z, b)
  const f2 dx = add2(t0.x, px), dy = add2(t0.y, py), dz = add2(t1.x, pz);
  const f2 r2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
  const f2 ir = rsqrt2(r2);
  const f2 ir2 = rcp2(r2);
  const f2 ir3 = mul2(ir2, ir);
  const f2 ad = fma2(t2.y, dz, fma2(t2.x, dy, mul2(t1.y, dx)));  // A.d
  acc[0] = fma2(ad, ir3, acc[0]);
  acc[0] = fma2(t4.y, ir, acc[0]);
  if (GRAD) {
    const f2 t = fma2(ad, mul2(ir2, pk(3.0f, 3.0f)), t4.y);  // 3 (A.d)/r^2 + b
    acc[1] = fma2(ir3, fma2(t, dx, t3.x), acc[1]);
    acc[2] = fma2(ir3, fma2(t, dy, t3.y), acc[2]);
    acc[3] = fma2(ir3, fma2(t, dz, t4.x), acc[3]);
  }
}

template <int D, bool GRAD>
__device__ __forceinline__ void pair_src(const ulonglong2* T, f2 px, f2 py, f2 pz, f2* acc) {
  const ulonglong2 t0 = T[0], t1 = T[1];
  if (D == 2) {
    // t0 = (y.x, y.y), t1 = (c ln2/(4 pi), -c/(2 pi))
    const f2 dx = add2(t0.x, px), dy = add2(t0.y, py);
    const f2 r2 = fma2(dy, dy, mul2(dx, dx));
    acc[0] = fma2(t1.x, lg22(r2), acc[0]);
    if (GRAD) {
      const f2 ci = mul2(t1.y, rcp2(r2));
      acc[1] = fma2(ci, dx, acc[1]);
      acc[2] = fma2(ci, dy, acc[2]);
    }
  } else {
    // t0 = (y.x, y.y), t1 = (y.z, -c/(4 pi))
    const f2 dx = add2(t0.x, px), dy = add2(t0.y, py), dz = add2(t1.x, pz);
    const f2 r2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
    const f2 ir = rsqrt2(r2);
    acc[0] = fma2(t1.y, ir, acc[0]);
    if (GRAD) {
      const f2 ci = mul2(t1.y, mul2(mul2(ir, ir), ir));
      acc[1] = fma2(ci, dx, acc[1]);
      acc[2] = fma2(ci, dy, acc[2]);
      acc[3] = fma2(ci, dz, acc[3]);
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

template <int D, int KIND, bool GRAD, int PTS>
__global__ void __launch_bounds__(kGBlock, GatherShape<PTS>::kMinBlocks) k_gather(const GatherArgs A) {
  constexpr int kGPts = GatherShape<PTS>::kPts;
  constexpr int kPtsPerCta = GatherShape<PTS>::kPtsPerCta;
  constexpr int SPF = KIND == 1 ? 2 : 5;
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

  // evaluation points of this thread (out-of-range points sit far away),
  // negated and packed two per register pair
  constexpr int NP = kGPts / 2;
  f2 px[NP], py[NP], pz[NP];
  int64_t kidx[kGPts];
#pragma unroll
  for (int j = 0; j < kGPts; ++j) kidx[j] = (int64_t)pb * kPtsPerCta + j * kGBlock + threadIdx.x;
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    float c[2][3];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int a = 0; a < 3; ++a)
        c[h][a] = (a < D && kidx[2 * j + h] < A.m) ? -A.x[a * A.m + kidx[2 * j + h]] : -(1.0e4f + (float)a);
    px[j] = pk(c[0][0], c[1][0]);
    py[j] = pk(c[0][1], c[1][1]);
    pz[j] = pk(c[0][2], c[1][2]);
  }
  constexpr bool SA = GatherShape<PTS>::kSmemAcc;
  __shared__ double sacc[SA ? kGPts * NA * kGBlock : 1];
  double acc64[SA ? 1 : kGPts][SA ? 1 : NA];
#pragma unroll
  for (int j = 0; j < kGPts; ++j)
#pragma unroll
    for (int q = 0; q < NA; ++q) {
      if (SA)
        sacc[(j * NA + q) * kGBlock + threadIdx.x] = 0.0;
      else
        acc64[SA ? 0 : j][SA ? 0 : q] = 0.0;
    }
  f2 acc[NP][NA];  // FP32 partial sums over kFlush tiles

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
      if (it % kFlush == 0)
#pragma unroll
        for (int j = 0; j < NP; ++j)
#pragma unroll
          for (int q = 0; q < NA; ++q) acc[j][q] = 0ull;
      const ulonglong2* T = reinterpret_cast<const ulonglong2*>(tile[b]);
#pragma unroll(D == 2 ? kUnroll2 : kUnroll3)
      for (int s = 0; s < cnt; ++s) {
        const ulonglong2* Ts = T + s * SPF;
#pragma unroll
        for (int j = 0; j < NP; ++j) {
          if (KIND == 1)
            pair_src<D, GRAD>(Ts, px[j], py[j], pz[j], acc[j]);
          else if (D == 2)
            pair_bnd2<GRAD>(Ts, px[j], py[j], acc[j]);
          else
            pair_bnd3<GRAD>(Ts, px[j], py[j], pz[j], acc[j]);
        }
      }
      if (it % kFlush == kFlush - 1 || it == nt - 1)
#pragma unroll
        for (int j = 0; j < NP; ++j)
#pragma unroll
          for (int q = 0; q < NA; ++q) {
            float lo, hi;
            upk(acc[j][q], lo, hi);
            if (SA) {
              sacc[((2 * j) * NA + q) * kGBlock + threadIdx.x] += (double)lo;
              sacc[((2 * j + 1) * NA + q) * kGBlock + threadIdx.x] += (double)hi;
            } else {
              acc64[SA ? 0 : 2 * j][SA ? 0 : q] += (double)lo;
              acc64[SA ? 0 : 2 * j + 1][SA ? 0 : q] += (double)hi;
            }
          }
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
        for (int q = 0; q < NA; ++q)
          A.out[q][k] += SA ? sacc[(j * NA + q) * kGBlock + threadIdx.x] : acc64[SA ? 0 : j][SA ? 0 : q];
    } else {
#pragma unroll
      for (int q = 0; q < NA; ++q)
        A.part[((int64_t)sp * NA + q) * A.m + k] =
            SA ? sacc[(j * NA + q) * kGBlock + threadIdx.x] : acc64[SA ? 0 : j][SA ? 0 : q];
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
  float4* o = (float4*)C.packed + 5 * i;
  const double ip = C.bnd_measure * (double)C.jac[i];  // 1/p of sample i
  if (D == 2) {
    const double a = C.u_hat[i] * ip / two_pi;
    const double b = C.dudn_hat[i] * ip / two_pi;
    const float zx = C.z[i], zy = C.z[C.n + i], nx = C.nrm[i], ny = C.nrm[C.n + i];
    const float fa = (float)a, fb = (float)b, a2 = (float)(2.0 * a), nbl = (float)(-b * 0.34657359027997265471);
    o[0] = make_float4(zx, zx, zy, zy);
    o[1] = make_float4(nx, nx, ny, ny);
    o[2] = make_float4(fa, fa, -fa, -fa);
    o[3] = make_float4(a2, a2, fb, fb);
    o[4] = make_float4(nbl, nbl, 0.0f, 0.0f);
  } else {
    const double a = C.u_hat[i] * ip / four_pi;
    const double b = C.dudn_hat[i] * ip / four_pi;
    const float zx = C.z[i], zy = C.z[C.n + i], zz = C.z[2 * C.n + i];
    const float ax = (float)(a * (double)C.nrm[i]), ay = (float)(a * (double)C.nrm[C.n + i]);
    const float az = (float)(a * (double)C.nrm[2 * C.n + i]), fb = (float)b;
    o[0] = make_float4(zx, zx, zy, zy);
    o[1] = make_float4(zz, zz, ax, ax);
    o[2] = make_float4(ay, ay, az, az);
    o[3] = make_float4(-ax, -ax, -ay, -ay);
    o[4] = make_float4(-az, -az, fb, fb);
  }
}

template <int D>
__global__ void __launch_bounds__(256) k_pack_src(const bvc_cache C) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= C.n_src_cand || j >= *C.n_src_dev) return;
  const double c = C.src_c[j];
  float4* o = (float4*)C.src_packed + 2 * j;
  const int64_t M = C.n_src_cand;
  const float yx = C.src_y[j], yy = C.src_y[M + j];
  o[0] = make_float4(yx, yx, yy, yy);
  if (D == 2) {
    const double c1 = c / 6.283185307179586476925;
    const float cl = (float)(c1 * 0.34657359027997265471), nc = (float)(-c1);
    o[1] = make_float4(cl, cl, nc, nc);
  } else {
    const float yz = C.src_y[2 * M + j], nc = (float)(-c / 12.566370614359172953850);
    o[1] = make_float4(yz, yz, nc, nc);
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

static Plan plan_gather(int pts, int64_t m, int64_t n, const void* kern) {
  Plan P;
  const int64_t per_cta = (int64_t)kGBlock * pts;
  P.pblocks = (int32_t)((m + per_cta - 1) / per_cta);
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
static const void* gather_kernel(int pts) {
  if (KIND == 1) return pts == 4 ? (const void*)k_gather<D, KIND, GRAD, 4> : (const void*)k_gather<D, KIND, GRAD, 2>;
  switch (pts) {
    case 2:
      return (const void*)k_gather<D, KIND, GRAD, 2>;
    case 4:
      return (const void*)k_gather<D, KIND, GRAD, 4>;
    default:
      return (const void*)k_gather<D, KIND, GRAD, 6>;
  }
}

static const void* pick(int D, int kind, bool grad, int pts) {
  if (D == 2) {
    if (kind == 0) return grad ? gather_kernel<2, 0, true>(pts) : gather_kernel<2, 0, false>(pts);
    return grad ? gather_kernel<2, 1, true>(pts) : gather_kernel<2, 1, false>(pts);
  }
  if (kind == 0) return grad ? gather_kernel<3, 0, true>(pts) : gather_kernel<3, 0, false>(pts);
  return grad ? gather_kernel<3, 1, true>(pts) : gather_kernel<3, 1, false>(pts);
}

static bool pts_supported(int kind, int pts) { return pts == 2 || pts == 4 || (kind == 0 && pts == 6); }

static size_t part_bytes(const Plan& P, int planes, int64_t m) {
  return P.n_splits > 1 ? (size_t)P.n_splits * planes * (size_t)m * sizeof(double) : 0;
}

// ---------------------------------------------------------------- screened
// Screened Poisson gather (App. A, sigma > 0, k = sqrt(sigma)): per sample
// the tile holds (z, A) and (n, B) with A = u^ |dOmega| / w, B = du/dn^
// |dOmega| / w, w = 2 pi (2D) or 4 pi (3D); with d = z - x, t = k r, the
// Green's functions G = -K0(t)/(2 pi) and -exp(-t)/(4 pi r) and
// Q = t K1(t) or exp(-t)(t + 1):
//   2D  u += A Q (n.d)/r^2 + B K0
//       grad u += A [Q (2 (n.d) d / r^4 - n / r^2) + (n.d)/r^2 k^2 K0 d] + B Q d / r^2
//   3D  u += A Q (n.d)/r^3 + B exp(-t)/r
//       grad u += A [Q (3 (n.d) d / r^5 - n / r^3) + (n.d)/r^3 k^2 exp(-t) d] + B Q d / r^3
// One point per thread, 128-sample tiles by bulk copy, FP32 per tile, FP64
// across tiles; sums added into the evaluation state like bvc_evaluate's.
// The same kernel serves the Poisson boundary term (SCR false: Q = 1, the
// K0 factor replaced by -ln r, exp(-t) by 1) when the u term's dG/dn is
// clamped to [-c, c] (Sec. 3.3, Eq. 9; CLAMP, cw = c w): the gradient terms
// stay unclamped.
constexpr int kSTile = 128;

template <int D>
__global__ void __launch_bounds__(256) k_pack_bnd_scr(const bvc_cache C) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= C.n) return;
  const double w = D == 2 ? 6.283185307179586476925 : 12.566370614359172953850;
  const double ca = C.bnd_measure * (double)C.jac[i] / w;
  float4* o = (float4*)C.packed + 2 * i;
  o[0] = make_float4(C.z[i], C.z[C.n + i], D == 3 ? C.z[2 * C.n + i] : 0.0f, (float)(C.u_hat[i] * ca));
  o[1] = make_float4(C.nrm[i], C.nrm[C.n + i], D == 3 ? C.nrm[2 * C.n + i] : 0.0f, (float)(C.dudn_hat[i] * ca));
}

// Source samples of a screened cache use the same tiles: (y, A = 0) and
// (0, B = -c / w), so that u += B K0 (2D) or B exp(-t)/r (3D) = G(x, y) c and
// grad u += B Q d / r^D = c dG/dx; n_dev (device) then holds the kept count.
template <int D>
__global__ void __launch_bounds__(256) k_pack_src_scr(const bvc_cache C) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= C.n_src_cand || j >= *C.n_src_dev) return;
  const int64_t M = C.n_src_cand;
  const double w = D == 2 ? 6.283185307179586476925 : 12.566370614359172953850;
  float4* o = (float4*)C.src_packed + 2 * j;
  o[0] = make_float4(C.src_y[j], C.src_y[M + j], D == 3 ? C.src_y[2 * M + j] : 0.0f, 0.0f);
  o[1] = make_float4(0.0f, 0.0f, 0.0f, (float)(-C.src_c[j] / w));
}

template <int D, bool GRAD, bool SCR, bool CLAMP>
__global__ void __launch_bounds__(256) k_gather_scr(const float* __restrict__ x, int64_t m, const float4* __restrict__ T,
                                                   int64_t n, const int64_t* __restrict__ n_dev, float k, float cw,
                                                   double* __restrict__ u, double* __restrict__ grad) {
  __shared__ __align__(128) float4 tile[2][2 * kSTile];
  __shared__ __align__(8) uint64_t bar[2];
  if (n_dev != nullptr) n = min64(n, *n_dev);
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  float pc[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) pc[a] = (a < D && p < m) ? x[a * m + p] : 1.0e4f + (float)a;
  double U = 0.0, Gd[3] = {0.0, 0.0, 0.0};
  const float k2 = k * k;
  const int64_t nt = (n + kSTile - 1) / kSTile;
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int b = 0; b < 2 && b < nt; ++b) {
      const uint32_t bytes = (uint32_t)min64(kSTile, n - (int64_t)b * kSTile) * 32u;
      mbar_expect_tx(&bar[b], bytes);
      bulk_g2s(&tile[b][0], T + 2 * (int64_t)b * kSTile, bytes, &bar[b]);
    }
  }
  for (int64_t it = 0; it < nt; ++it) {
    const int b = (int)(it & 1);
    const bool ok = mbar_wait_bounded(&bar[b], (uint32_t)((it >> 1) & 1));
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {
        atomicOr(&g_gather_status, 1ull);
        for (int64_t k3 = it; k3 < it + 2 && k3 < nt; ++k3)
          (void)mbar_wait_bounded(&bar[k3 & 1], (uint32_t)((k3 >> 1) & 1));
      }
      return;
    }
    const int cnt = (int)min64(kSTile, n - it * kSTile);
    float au = 0.0f, ag[3] = {0.0f, 0.0f, 0.0f};
    for (int e = 0; e < cnt; ++e) {
      const float4 zA = tile[b][2 * e], nB = tile[b][2 * e + 1];
      const float dx = zA.x - pc[0], dy = zA.y - pc[1], dz = D == 3 ? zA.z - pc[2] : 0.0f;
      const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
      const float ir = rsqrtf(r2), r = r2 * ir, t = k * r;
      const float nd = fmaf(nB.z, dz, fmaf(nB.y, dy, nB.x * dx));
      float Q, kern, dq;  // Q; K0 or exp(-t)/r; the gradient factor of Q
      float ik;           // 1/r^2 (2D) or 1/r^3 (3D)
      if (!SCR) {
        Q = 1.0f;
        dq = 0.0f;
        kern = D == 2 ? -0.5f * __logf(r2) : ir;
        ik = D == 2 ? ir * ir : ir * ir * ir;
      } else if (D == 2) {
        float k0, k1;
        if (t <= 2.0f) {
          k0 = bessel_k0_small(t);
          k1 = bessel_k1_small(t);
        } else {
          const float e2 = __expf(-t) * rsqrtf(t);
          k0 = bessel_k0s_large(t) * e2;
          k1 = bessel_k1s_large(t) * e2;
        }
        Q = t * k1;
        kern = k0;
        dq = k2 * k0;
        ik = ir * ir;
      } else {
        const float e3 = __expf(-t);
        Q = e3 * (t + 1.0f);
        kern = e3 * ir;
        dq = k2 * e3;
        ik = ir * ir * ir;
      }
      const float s1 = CLAMP ? zA.w * fminf(fmaxf(Q * nd * ik, -cw), cw) : zA.w * Q * nd * ik;
      au += fmaf(nB.w, kern, s1);
      if (GRAD) {
        // A [Q (D (n.d) d / r^(D+2) - n / r^D) + (n.d)/r^D dq d] + B Q d / r^D
        const float c1 = zA.w * (Q * (float)D * nd * ik * ir * ir + nd * ik * dq) + nB.w * Q * ik;
        const float c2 = -zA.w * Q * ik;
        ag[0] = fmaf(c1, dx, fmaf(c2, nB.x, ag[0]));
        ag[1] = fmaf(c1, dy, fmaf(c2, nB.y, ag[1]));
        if (D == 3) ag[2] = fmaf(c1, dz, fmaf(c2, nB.z, ag[2]));
      }
    }
    U += (double)au;
    if (GRAD) {
#pragma unroll
      for (int a = 0; a < D; ++a) Gd[a] += (double)ag[a];
    }
    __syncthreads();
    if (threadIdx.x == 0 && it + 2 < nt) {
      fence_proxy_async();
      const int64_t st = (it + 2) * kSTile;
      const uint32_t bytes = (uint32_t)min64(kSTile, n - st) * 32u;
      mbar_expect_tx(&bar[b], bytes);
      bulk_g2s(&tile[b][0], T + 2 * st, bytes, &bar[b]);
    }
  }
  if (p < m) {
    u[p] += U;
    if (GRAD) {
#pragma unroll
      for (int a = 0; a < D; ++a) grad[a * m + p] += Gd[a];
    }
  }
}

}  // namespace bvc

using namespace bvc;

static bvc_status bvc_cache_pack_impl(const bvc_cache* cache, bvc_stream stream) {
  if (cache == nullptr || (cache->dim != 2 && cache->dim != 3) || cache->n < 0) return BVC_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (cache->n > 0) {
    if (!cache->z || !cache->nrm || !cache->jac || !cache->u_hat || !cache->dudn_hat || !cache->packed)
      return BVC_ERR_INVALID_ARG;
    const unsigned grid = (unsigned)((cache->n + 255) / 256);
    ProfScope ps("pack_boundary", s);
    if (cache->sigma > 0.0 || cache->clamp_c > 0.0) {
      if (cache->dim == 2)
        k_pack_bnd_scr<2><<<grid, 256, 0, s>>>(*cache);
      else
        k_pack_bnd_scr<3><<<grid, 256, 0, s>>>(*cache);
    } else if (cache->dim == 2) {
      k_pack_bnd<2><<<grid, 256, 0, s>>>(*cache);
    } else {
      k_pack_bnd<3><<<grid, 256, 0, s>>>(*cache);
    }
  }
  if (cache->n_src_cand > 0) {
    if (!cache->src_y || !cache->src_c || !cache->src_packed || !cache->n_src_dev) return BVC_ERR_INVALID_ARG;
    const unsigned grid = (unsigned)((cache->n_src_cand + 255) / 256);
    ProfScope ps("pack_source", s);
    if (cache->sigma > 0.0) {  // the screened gather's tile layout
      if (cache->dim == 2)
        k_pack_src_scr<2><<<grid, 256, 0, s>>>(*cache);
      else
        k_pack_src_scr<3><<<grid, 256, 0, s>>>(*cache);
    } else if (cache->dim == 2) {
      k_pack_src<2><<<grid, 256, 0, s>>>(*cache);
    } else {
      k_pack_src<3><<<grid, 256, 0, s>>>(*cache);
    }
  }
  BVC_LAUNCH_CHECK();
  return BVC_OK;
}
extern "C" bvc_status bvc_cache_pack(const bvc_cache* cache, bvc_stream stream) {
  return bvc::note_status(bvc_cache_pack_impl(cache, stream));
}

static bvc_status bvc_evaluate_workspace_size_impl(const bvc_cache* cache, const bvc_eval_state* state,
                                                  size_t* bytes) {
  if (cache == nullptr || state == nullptr || bytes == nullptr || cache->dim != state->dim) return BVC_ERR_INVALID_ARG;
  const int D = cache->dim;
  const bool grad = state->grad_bnd != nullptr;
  const int planes = grad ? 1 + D : 1;
  // the largest over the supported points-per-thread counts, so that any
  // shape bvc_tune_gather picks fits
  size_t b = 0;
  for (int pts = 2; pts <= 6; pts += 2) {
    if (cache->n > 0) {
      const size_t bb = part_bytes(plan_gather(pts, state->m, cache->n, pick(D, 0, grad, pts)), planes, state->m);
      b = bb > b ? bb : b;
    }
    if (cache->n_src_cand > 0 && pts_supported(1, pts)) {
      const Plan P = plan_gather(pts, state->m, cache->n_src_cand, pick(D, 1, grad, pts));
      const size_t bs = part_bytes(P, planes, state->m);
      b = bs > b ? bs : b;
    }
  }
  *bytes = b;
  return BVC_OK;
}
extern "C" bvc_status bvc_evaluate_workspace_size(const bvc_cache* cache, const bvc_eval_state* state,
                                                  size_t* bytes) {
  return bvc::note_status(bvc_evaluate_workspace_size_impl(cache, state, bytes));
}

static bvc_status run_part(int D, int kind, bool grad, const float* x, int64_t m, const float4* samples, int64_t n,
                           const int64_t* n_dev, double* u, double* g, void* ws, size_t ws_bytes, cudaStream_t s,
                           int pts = 0) {
  if (pts == 0) pts = gather_pts(D, kind);
  const void* kern = pick(D, kind, grad, pts);
  const Plan P = plan_gather(pts, m, n, kern);
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

static bvc_status bvc_evaluate_impl(const bvc_cache* cache, bvc_eval_state* state, void* workspace,
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
    if (cache->n > 0 && (cache->sigma > 0.0 || cache->clamp_c > 0.0)) {
      const unsigned grid = (unsigned)((state->m + 255) / 256);
      const float k = (float)sqrt(cache->sigma);
      const float cw = (float)(cache->clamp_c * (D == 2 ? 6.283185307179586476925 : 12.566370614359172953850));
      const bool scr = cache->sigma > 0.0, clamp = cache->clamp_c > 0.0;
      const float4* T = (const float4*)cache->packed;
      ProfScope ps(scr ? "gather_screened" : "gather_clamped", s);
#define BVC_FLEX(DD, GG, SS, CC) \
  k_gather_scr<DD, GG, SS, CC><<<grid, 256, 0, s>>>(state->x, state->m, T, cache->n, nullptr, k, cw, state->u_bnd, \
                                                    GG ? state->grad_bnd : nullptr)
#define BVC_FLEX_D(DD) \
  if (grad) {                                                  \
    if (scr) {                                                 \
      if (clamp) BVC_FLEX(DD, true, true, true);               \
      else BVC_FLEX(DD, true, true, false);                    \
    } else {                                                   \
      BVC_FLEX(DD, true, false, true);                         \
    }                                                          \
  } else {                                                     \
    if (scr) {                                                 \
      if (clamp) BVC_FLEX(DD, false, true, true);              \
      else BVC_FLEX(DD, false, true, false);                   \
    } else {                                                   \
      BVC_FLEX(DD, false, false, true);                        \
    }                                                          \
  }
      if (D == 2) {
        BVC_FLEX_D(2)
      } else {
        BVC_FLEX_D(3)
      }
#undef BVC_FLEX_D
#undef BVC_FLEX
      BVC_LAUNCH_CHECK();
    } else if (cache->n > 0) {
      bvc_status st = run_part(D, 0, grad, state->x, state->m, (const float4*)cache->packed, cache->n, nullptr,
                               state->u_bnd, state->grad_bnd, workspace, workspace_bytes, s);
      if (st != BVC_OK) return st;
    }
    if (cache->n_src_cand > 0 && cache->sigma > 0.0) {
      // screened source samples: G^sigma(x, y) c through the screened gather
      const unsigned grid = (unsigned)((state->m + 255) / 256);
      const float k = (float)sqrt(cache->sigma);
      const float4* T = (const float4*)cache->src_packed;
      ProfScope ps("gather_screened_source", s);
      if (D == 2) {
        if (grad)
          k_gather_scr<2, true, true, false><<<grid, 256, 0, s>>>(state->x, state->m, T, cache->n_src_cand,
                                                                  cache->n_src_dev, k, 0.0f, state->u_src,
                                                                  state->grad_src);
        else
          k_gather_scr<2, false, true, false><<<grid, 256, 0, s>>>(state->x, state->m, T, cache->n_src_cand,
                                                                   cache->n_src_dev, k, 0.0f, state->u_src, nullptr);
      } else {
        if (grad)
          k_gather_scr<3, true, true, false><<<grid, 256, 0, s>>>(state->x, state->m, T, cache->n_src_cand,
                                                                  cache->n_src_dev, k, 0.0f, state->u_src,
                                                                  state->grad_src);
        else
          k_gather_scr<3, false, true, false><<<grid, 256, 0, s>>>(state->x, state->m, T, cache->n_src_cand,
                                                                   cache->n_src_dev, k, 0.0f, state->u_src, nullptr);
      }
      BVC_LAUNCH_CHECK();
    } else if (cache->n_src_cand > 0) {
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
extern "C" bvc_status bvc_evaluate(const bvc_cache* cache, bvc_eval_state* state, void* workspace,
                                   size_t workspace_bytes, bvc_stream stream) {
  return bvc::note_status(bvc_evaluate_impl(cache, state, workspace, workspace_bytes, stream));
}

// The gather autotuner: for each kind of samples the cache has (boundary
// with the plain Poisson kernel, sources), times two launches of every
// supported points-per-thread count on this cache and these points and
// keeps the fastest for all later gathers of that dimension and kind.
static bvc_status bvc_tune_gather_impl(const bvc_cache* cache, bvc_eval_state* state, void* workspace,
                                      size_t workspace_bytes, bvc_stream stream, int32_t pts_out[2],
                                      float* best_ms) {
  if (cache == nullptr || state == nullptr || cache->dim != state->dim || (cache->dim != 2 && cache->dim != 3) ||
      state->m < 1 || state->x == nullptr || state->u_bnd == nullptr || state->u_src == nullptr ||
      state->counts == nullptr || pts_out == nullptr)
    return BVC_ERR_INVALID_ARG;
  const int D = cache->dim;
  const bool grad = state->grad_bnd != nullptr;
  if (grad != (state->grad_src != nullptr)) return BVC_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  BVC_CUDA_TRY(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return BVC_ERR_CUDA;
  }
  bvc_status st = BVC_OK;
  float total = 0.0f;
  for (int kind = 0; kind < 2 && st == BVC_OK; ++kind) {
    pts_out[kind] = gather_pts(D, kind);
    const bool have = kind == 0 ? (cache->n > 0 && cache->packed != nullptr && cache->sigma == 0.0 &&
                                   cache->clamp_c == 0.0)
                                : (cache->n_src_cand > 0 && cache->src_packed != nullptr && cache->n_src_dev != nullptr &&
                                   cache->sigma == 0.0);
    if (!have) continue;
    const float4* T = (const float4*)(kind == 0 ? cache->packed : cache->src_packed);
    const int64_t n = kind == 0 ? cache->n : cache->n_src_cand;
    const int64_t* nd = kind == 0 ? nullptr : cache->n_src_dev;
    float best = INFINITY;
    int best_pts = pts_out[kind];
    for (int pts = 2; pts <= 6 && st == BVC_OK; pts += 2) {
      if (!pts_supported(kind, pts)) continue;
      for (int rep = 0; rep < 2 && st == BVC_OK; ++rep) {
        if (cudaEventRecord(e0, s) != cudaSuccess) st = BVC_ERR_CUDA;
        if (st == BVC_OK)
          st = run_part(D, kind, grad, state->x, state->m, T, n, nd, kind == 0 ? state->u_bnd : state->u_src,
                        kind == 0 ? state->grad_bnd : state->grad_src, workspace, workspace_bytes, s, pts);
        float ms = 0.0f;
        if (st == BVC_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                             cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
          st = BVC_ERR_CUDA;
        if (st == BVC_OK && ms < best) {
          best = ms;
          best_pts = pts;
        }
      }
    }
    if (st == BVC_OK) {
      __atomic_store_n(&g_gather_pts[D - 2][kind], best_pts, __ATOMIC_RELAXED);
      pts_out[kind] = best_pts;
      total += best;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != BVC_OK) return st;
  if (best_ms) *best_ms = total;
  return bvc_eval_state_reset(state, stream);
}
extern "C" bvc_status bvc_tune_gather(const bvc_cache* cache, bvc_eval_state* state, void* workspace,
                                      size_t workspace_bytes, bvc_stream stream, int32_t pts_out[2],
                                      float* best_ms) {
  return bvc::note_status(bvc_tune_gather_impl(cache, state, workspace, workspace_bytes, stream, pts_out, best_ms));
}

static bvc_status bvc_set_gather_shape_impl(int32_t dim, int32_t kind, int32_t pts) {
  if ((dim != 2 && dim != 3) || (kind != 0 && kind != 1) || (pts != 0 && !pts_supported(kind, pts)))
    return BVC_ERR_INVALID_ARG;
  __atomic_store_n(&g_gather_pts[dim - 2][kind], pts, __ATOMIC_RELAXED);
  return BVC_OK;
}
extern "C" bvc_status bvc_set_gather_shape(int32_t dim, int32_t kind, int32_t pts) {
  return bvc::note_status(bvc_set_gather_shape_impl(dim, kind, pts));
}

static bvc_status bvc_eval_state_reset_impl(const bvc_eval_state* state, bvc_stream stream) {
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
extern "C" bvc_status bvc_eval_state_reset(const bvc_eval_state* state, bvc_stream stream) {
  return bvc::note_status(bvc_eval_state_reset_impl(state, stream));
}

static bvc_status bvc_get_solution_impl(const bvc_eval_state* state, double* u, double* grad, bvc_stream stream) {
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
extern "C" bvc_status bvc_get_solution(const bvc_eval_state* state, double* u, double* grad, bvc_stream stream) {
  return bvc::note_status(bvc_get_solution_impl(state, u, grad, stream));
}

// Self-test of the bounded wait: one warp waits on a barrier that nothing
// completes; the wait gives up after limit_ns and the status word records it
// (bit 1), as a stalled tile copy would (bit 0).
__global__ void k_wait_selftest(uint64_t limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncwarp();
  const bool ok = mbar_wait_bounded_ns(&bar, 0u, limit_ns);
  if (!ok && threadIdx.x == 0) atomicOr(&g_gather_status, 2ull);
}

static bvc_status bvc_wait_selftest_impl(int64_t limit_ns, bvc_stream stream) {
  if (limit_ns < 0 || limit_ns > 2000000000ll) return BVC_ERR_INVALID_ARG;
  k_wait_selftest<<<1, 32, 0, (cudaStream_t)stream>>>((uint64_t)limit_ns);
  BVC_LAUNCH_CHECK();
  return BVC_OK;
}
extern "C" bvc_status bvc_wait_selftest(int64_t limit_ns, bvc_stream stream) {
  return bvc::note_status(bvc_wait_selftest_impl(limit_ns, stream));
}

static bvc_status bvc_gather_status_impl(uint64_t* flags, int32_t reset) {
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
extern "C" bvc_status bvc_gather_status(uint64_t* flags, int32_t reset) {
  return bvc::note_status(bvc_gather_status_impl(flags, reset));
}

// ---------------------------------------------------------------------------
// Eq. 3 for many right-hand sides: per pair the two kernel values
// (2D: (n.d)/r^2 and lg2 r^2; 3D: (n.d)/r^3 and 1/r) are computed once and
// applied to the BVC_MULTI_GROUP coefficient pairs of the tile's samples.
// One thread per evaluation point, 32 FP32 partial sums flushed to FP64
// every tile of 32 samples; tiles staged by bulk asynchronous copies.
namespace bvc {

constexpr int kMG = BVC_MULTI_GROUP;
constexpr int kMTile = 32;
// FP32 partial sums cover kMFlush tiles (128 samples) before they are added
// to the FP64 sums: GB300's FP64 pipe runs at 1/64 of the FP32 rate, and one
// FP64 add per right-hand side every 32 samples would occupy it almost as
// long as the FP32 work itself.
constexpr int kMFlush = 4;
constexpr int kMStride = 8 + 2 * kMG;  // floats per packed sample row

// One mesh (meshes == null): m points [D][m] against n samples, then (a
// cache with a source) the *extra kept source rows (at most n_extra) that
// follow them in each group's block of rows_g rows; the sums are divided by
// n either way (the source rows carry the factor n/M).  A batch:
// block x belongs to the mesh whose gather blocks hold it; its points lie in
// that mesh's range of the [D][m] point planes and its samples in that
// mesh's range of the n sample rows of each group.
//
// 128 threads, two points each (a block covers 256 points): every sample's
// 32 coefficient pairs, broadcast from shared memory, feed both points, which
// halves the shared-memory reads per FMA.  The 64 FP32 partial sums of a
// thread live in registers, two right-hand sides per packed FP32x2 register
// pair (the coefficients of adjacent right-hand sides are adjacent in the
// tile, so each fma.rn.f32x2 updates two sums: the same rounding as two
// fmaf, half the issue slots); the FP64 running sums in shared memory
// (dynamic, kMSum64 bytes), column per thread.
constexpr int kMThreads = 128;
constexpr int kMSum64 = 2 * kMG * kMThreads * 8;

template <int D>
__global__ void __launch_bounds__(kMThreads, 2) k_gather_multi(const float* __restrict__ x, int64_t m,
                                                               const float* __restrict__ packed, int64_t n, int32_t K,
                                                               double* __restrict__ u,
                                                               const BatchMeshDev* __restrict__ meshes,
                                                               int32_t count, int64_t rows_g,
                                                               const int64_t* __restrict__ extra, int64_t n_extra) {
  __shared__ __align__(128) float tile[2][kMTile * kMStride];
  __shared__ __align__(8) uint64_t bar[2];
  extern __shared__ double s64[];  // [2 * kMG][kMThreads]
  const int g = blockIdx.y;
  const int tid = threadIdx.x;
  int64_t blk = blockIdx.x, pt_off = 0, n_pts = m, smp_off = 0, n_smp = n;
  if (meshes != nullptr) {
    int lo = 0, hi = count - 1;  // the last mesh whose first block is <= blockIdx.x
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (meshes[mid].blk_off <= (int64_t)blockIdx.x)
        lo = mid;
      else
        hi = mid - 1;
    }
    const BatchMeshDev M = meshes[lo];
    blk -= M.blk_off;
    pt_off = M.pt_off;
    n_pts = M.n_pts;
    smp_off = M.smp_off;
    n_smp = M.n_smp;
  }
  const float* base = packed + ((int64_t)g * rows_g + smp_off) * kMStride;
  int64_t n_rows = n_smp;
  if (extra != nullptr) n_rows += min64(*extra, n_extra);
  const int64_t pl0 = blk * (2 * kMThreads) + tid, pl1 = pl0 + kMThreads;  // points within the mesh
  float pa[3], pb[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    pa[a] = (a < D && pl0 < n_pts) ? x[a * m + pt_off + pl0] : 1.0e4f + (float)a;
    pb[a] = (a < D && pl1 < n_pts) ? x[a * m + pt_off + pl1] : 1.0e4f + (float)a;
  }
  f2 acc0[kMG / 2], acc1[kMG / 2];  // (right-hand side 2h, 2h + 1) of the two points
#pragma unroll
  for (int q = 0; q < 2 * kMG; ++q) s64[q * kMThreads + tid] = 0.0;
  const int64_t nt = (n_rows + kMTile - 1) / kMTile;
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0) {
    for (int b = 0; b < 2 && b < nt; ++b) {
      const int64_t st = (int64_t)b * kMTile;
      const uint32_t bytes = (uint32_t)min64(kMTile, n_rows - st) * kMStride * 4u;
      mbar_expect_tx(&bar[b], bytes);
      bulk_g2s(&tile[b][0], base + st * kMStride, bytes, &bar[b]);
    }
  }
  for (int64_t it = 0; it < nt; ++it) {
    const int b = (int)(it & 1);
    const bool ok = mbar_wait_bounded(&bar[b], (uint32_t)((it >> 1) & 1));
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicOr(&g_gather_status, 1ull);
        for (int64_t k2 = it; k2 < it + 2 && k2 < nt; ++k2)
          (void)mbar_wait_bounded(&bar[k2 & 1], (uint32_t)((k2 >> 1) & 1));
      }
      return;
    }
    const int cnt = (int)min64(kMTile, n_rows - it * kMTile);
    if (it % kMFlush == 0) {
#pragma unroll
      for (int q = 0; q < kMG / 2; ++q) acc0[q] = acc1[q] = 0ull;
    }
    const float4* T = reinterpret_cast<const float4*>(tile[b]);
    for (int s = 0; s < cnt; ++s) {
      const float4* row = T + s * (kMStride / 4);
      const float4 zz = row[0], nn = row[1];
      float ka1, ka2, kb1, kb2;
      {
        const float dx = zz.x - pa[0], dy = zz.y - pa[1], dz = zz.z - pa[2];
        if (D == 2) {
          const float r2 = fmaf(dy, dy, dx * dx);
          ka1 = fmaf(nn.y, dy, nn.x * dx) * rcp_approx(r2);
          ka2 = lg2_approx(r2);
        } else {
          const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
          const float ir = rsqrt_approx(r2);
          ka1 = fmaf(nn.z, dz, fmaf(nn.y, dy, nn.x * dx)) * (ir * ir * ir);
          ka2 = ir;
        }
      }
      {
        const float dx = zz.x - pb[0], dy = zz.y - pb[1], dz = zz.z - pb[2];
        if (D == 2) {
          const float r2 = fmaf(dy, dy, dx * dx);
          kb1 = fmaf(nn.y, dy, nn.x * dx) * rcp_approx(r2);
          kb2 = lg2_approx(r2);
        } else {
          const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
          const float ir = rsqrt_approx(r2);
          kb1 = fmaf(nn.z, dz, fmaf(nn.y, dy, nn.x * dx)) * (ir * ir * ir);
          kb2 = ir;
        }
      }
      const f2 ka1p = pk(ka1, ka1), ka2p = pk(ka2, ka2), kb1p = pk(kb1, kb1), kb2p = pk(kb2, kb2);
      const ulonglong2* R2 = reinterpret_cast<const ulonglong2*>(row);
#pragma unroll
      for (int q = 0; q < kMG / 4; ++q) {
        const ulonglong2 a4 = R2[2 + q], b4 = R2[2 + kMG / 4 + q];
        acc0[2 * q + 0] = fma2(b4.x, ka2p, fma2(a4.x, ka1p, acc0[2 * q + 0]));
        acc0[2 * q + 1] = fma2(b4.y, ka2p, fma2(a4.y, ka1p, acc0[2 * q + 1]));
        acc1[2 * q + 0] = fma2(b4.x, kb2p, fma2(a4.x, kb1p, acc1[2 * q + 0]));
        acc1[2 * q + 1] = fma2(b4.y, kb2p, fma2(a4.y, kb1p, acc1[2 * q + 1]));
      }
    }
    if (it % kMFlush == kMFlush - 1 || it == nt - 1) {
#pragma unroll
      for (int q = 0; q < kMG / 2; ++q) {
        float a_lo, a_hi, b_lo, b_hi;
        upk(acc0[q], a_lo, a_hi);
        upk(acc1[q], b_lo, b_hi);
        s64[(2 * q) * kMThreads + tid] += (double)a_lo;
        s64[(2 * q + 1) * kMThreads + tid] += (double)a_hi;
        s64[(kMG + 2 * q) * kMThreads + tid] += (double)b_lo;
        s64[(kMG + 2 * q + 1) * kMThreads + tid] += (double)b_hi;
      }
    }
    __syncthreads();
    if (tid == 0 && it + 2 < nt) {
      fence_proxy_async();
      const int64_t st = (it + 2) * kMTile;
      const uint32_t bytes = (uint32_t)min64(kMTile, n_rows - st) * kMStride * 4u;
      mbar_expect_tx(&bar[b], bytes);
      bulk_g2s(&tile[b][0], base + st * kMStride, bytes, &bar[b]);
    }
  }
  const int kk = (K - g * kMG) < kMG ? (K - g * kMG) : kMG;
  const double inv_n = 1.0 / (double)n_smp;
  for (int h = 0; h < 2; ++h) {
    const int64_t pl = h ? pl1 : pl0;
    if (pl >= n_pts) continue;
    for (int q = 0; q < kk; ++q) u[(int64_t)(g * kMG + q) * m + pt_off + pl] = s64[(h * kMG + q) * kMThreads + tid] * inv_n;
  }
}

// The dynamic shared memory of k_gather_multi exceeds the default 48 KB.
template <int D>
static bvc_status multi_gather_attr() {
  static bool done = false;
  if (!done) {
    if (cudaFuncSetAttribute((const void*)k_gather_multi<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMSum64) !=
        cudaSuccess) {
      (void)cudaGetLastError();
      return BVC_ERR_CUDA;
    }
    done = true;
  }
  return BVC_OK;
}

// ---------------------------------------------------------------- adjoint
// Eq. 3 transposed: with lam(x) = dL/du(x) at the evaluation points,
//   boundary sample i:  S1_i = sum_x lam(x) K1(x, z_i),  S2_i = sum_x lam(x) K2(x, z_i)
//   source sample j:    S_j  = sum_x lam(x) G'(x, y_j)
// with the gather's kernels (2D K1 = n.d / r^2, K2 = lg2 r^2; 3D K1 = n.d /
// r^3, K2 = 1/r; G' = lg2 r^2 (2D), 1/r (3D)); the host scales them into
// dL/du^, dL/d(du/dn^) and dL/dc.  Points, packed (x, lam) as float4, are
// staged in shared memory by bulk copies, double-buffered; each thread owns
// kAS samples.  FP32 sums per tile of kATile points, FP64 across tiles.
constexpr int kATile = 128;
constexpr int kAS = 4;

template <int D, bool SRC>
__global__ void __launch_bounds__(256) k_gather_adj(const float4* __restrict__ pl, int64_t m,
                                                   const float* __restrict__ zs, const float* __restrict__ ns,
                                                   const float* __restrict__ jw, int64_t stride,
                                                   const int64_t* __restrict__ n_dev, int64_t n_fix, double s1,
                                                   double s2, double* __restrict__ out1, double* __restrict__ out2) {
  __shared__ __align__(128) float4 tile[2][kATile];
  __shared__ __align__(8) uint64_t bar[2];
  const int64_t n = n_dev ? *n_dev : n_fix;
  const int64_t base = (int64_t)blockIdx.x * blockDim.x * kAS;
  if (base >= n) return;  // whole block idle (uniform)
  float zc[kAS][3], nc[kAS][3];
  bool live[kAS];
#pragma unroll
  for (int q = 0; q < kAS; ++q) {
    const int64_t i = base + (int64_t)q * blockDim.x + threadIdx.x;
    live[q] = i < n;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      zc[q][a] = (a < D && live[q]) ? zs[a * stride + i] : 0.0f;
      nc[q][a] = (!SRC && a < D && live[q]) ? ns[a * stride + i] : 0.0f;
    }
  }
  double A1[kAS], A2[kAS];
#pragma unroll
  for (int q = 0; q < kAS; ++q) A1[q] = A2[q] = 0.0;
  const int64_t nt = (m + kATile - 1) / kATile;
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int b = 0; b < 2 && b < nt; ++b) {
      const uint32_t bytes = (uint32_t)min64(kATile, m - (int64_t)b * kATile) * 16u;
      mbar_expect_tx(&bar[b], bytes);
      bulk_g2s(&tile[b][0], pl + (int64_t)b * kATile, bytes, &bar[b]);
    }
  }
  for (int64_t it = 0; it < nt; ++it) {
    const int b = (int)(it & 1);
    const bool ok = mbar_wait_bounded(&bar[b], (uint32_t)((it >> 1) & 1));
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {
        atomicOr(&g_gather_status, 1ull);
        for (int64_t k2 = it; k2 < it + 2 && k2 < nt; ++k2)
          (void)mbar_wait_bounded(&bar[k2 & 1], (uint32_t)((k2 >> 1) & 1));
      }
      return;
    }
    const int cnt = (int)min64(kATile, m - it * kATile);
    float a1[kAS], a2[kAS];
#pragma unroll
    for (int q = 0; q < kAS; ++q) a1[q] = a2[q] = 0.0f;
    for (int e = 0; e < cnt; ++e) {
      const float4 P = tile[b][e];  // (x, y, z, lam)
#pragma unroll
      for (int q = 0; q < kAS; ++q) {
        const float dx = zc[q][0] - P.x, dy = zc[q][1] - P.y, dz = D == 3 ? zc[q][2] - P.z : 0.0f;
        const float r2 = D == 3 ? fmaf(dz, dz, fmaf(dy, dy, dx * dx)) : fmaf(dy, dy, dx * dx);
        if (D == 2) {
          const float l2 = lg2_approx(r2);
          if (SRC) {
            a1[q] = fmaf(P.w, l2, a1[q]);
          } else {
            const float k1 = fmaf(nc[q][1], dy, nc[q][0] * dx) * rcp_approx(r2);
            a1[q] = fmaf(P.w, k1, a1[q]);
            a2[q] = fmaf(P.w, l2, a2[q]);
          }
        } else {
          const float ir = rsqrt_approx(r2);
          if (SRC) {
            a1[q] = fmaf(P.w, ir, a1[q]);
          } else {
            const float k1 = fmaf(nc[q][2], dz, fmaf(nc[q][1], dy, nc[q][0] * dx)) * (ir * ir * ir);
            a1[q] = fmaf(P.w, k1, a1[q]);
            a2[q] = fmaf(P.w, ir, a2[q]);
          }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < kAS; ++q) {
      A1[q] += (double)a1[q];
      A2[q] += (double)a2[q];
    }
    __syncthreads();
    if (threadIdx.x == 0 && it + 2 < nt) {
      fence_proxy_async();
      const int64_t st = (it + 2) * kATile;
      const uint32_t bytes = (uint32_t)min64(kATile, m - st) * 16u;
      mbar_expect_tx(&bar[b], bytes);
      bulk_g2s(&tile[b][0], pl + st, bytes, &bar[b]);
    }
  }
#pragma unroll
  for (int q = 0; q < kAS; ++q) {
    if (!live[q]) continue;
    const int64_t i = base + (int64_t)q * blockDim.x + threadIdx.x;
    const double wi = jw != nullptr ? (double)jw[i] : 1.0;  // per-sample 1/p factor
    out1[i] = A1[q] * s1 * wi;
    if (!SRC) out2[i] = A2[q] * s2 * wi;
  }
}

template <int D>
__global__ void __launch_bounds__(256) k_pack_adj_pts(const float* __restrict__ x, int64_t m,
                                                     const double* __restrict__ lam, float4* __restrict__ out) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= m) return;
  out[p] = make_float4(x[p], x[m + p], D == 3 ? x[2 * m + p] : 0.0f, (float)lam[p]);
}

}  // namespace bvc

static bvc_status bvc_evaluate_multi_impl(const bvc_multi_cache* cache, const float* pts, int64_t m, double* u,
                                         bvc_stream stream) {
  if (cache == nullptr || (cache->dim != 2 && cache->dim != 3) || cache->n < 1 || cache->k < 1 ||
      cache->packed == nullptr || m < 0 || (m > 0 && (pts == nullptr || u == nullptr)))
    return BVC_ERR_INVALID_ARG;
  const int groups = (cache->k + kMG - 1) / kMG;
  if (groups > 65535) return BVC_ERR_INVALID_ARG;  // grid.y limit
  const int64_t M = cache->n_src_cand > 0 ? cache->n_src_cand : 0;
  if (M > 0 && cache->n_src_dev == nullptr) return BVC_ERR_INVALID_ARG;
  const int64_t rows = cache->n + M;
  const int64_t* extra = M > 0 ? cache->n_src_dev : nullptr;
  if (m == 0) return BVC_OK;
  const dim3 grid((unsigned)((m + 255) / 256), (unsigned)groups);
  cudaStream_t s = (cudaStream_t)stream;
  ProfScope ps("gather_multi", s);
  const bvc_status at = cache->dim == 2 ? multi_gather_attr<2>() : multi_gather_attr<3>();
  if (at != BVC_OK) return at;
  if (cache->dim == 2)
    k_gather_multi<2><<<grid, kMThreads, kMSum64, s>>>(pts, m, cache->packed, cache->n, cache->k, u, nullptr, 0,
                                                       rows, extra, M);
  else
    k_gather_multi<3><<<grid, kMThreads, kMSum64, s>>>(pts, m, cache->packed, cache->n, cache->k, u, nullptr, 0,
                                                       rows, extra, M);
  BVC_LAUNCH_CHECK();
  return BVC_OK;
}
extern "C" bvc_status bvc_evaluate_multi(const bvc_multi_cache* cache, const float* pts, int64_t m, double* u,
                                         bvc_stream stream) {
  return bvc::note_status(bvc_evaluate_multi_impl(cache, pts, m, u, stream));
}

static bvc_status bvc_batch_evaluate_impl(bvc_batch b, const bvc_multi_cache* cache, const float* pts, double* u,
                                         bvc_stream stream) {
  if (b == nullptr || cache == nullptr || cache->dim != b->dim || cache->n != b->n_total || cache->k != b->k ||
      cache->packed == nullptr || cache->n_src_cand != 0 || (b->m_total > 0 && (pts == nullptr || u == nullptr)))
    return BVC_ERR_INVALID_ARG;
  const int groups = (cache->k + kMG - 1) / kMG;
  if (groups > 65535 || b->blocks_total > 0x7fffffffLL) return BVC_ERR_INVALID_ARG;  // grid limits
  if (b->blocks_total == 0) return BVC_OK;
  const dim3 grid((unsigned)b->blocks_total, (unsigned)groups);
  cudaStream_t s = (cudaStream_t)stream;
  ProfScope ps("gather_multi", s);
  const bvc_status at = b->dim == 2 ? multi_gather_attr<2>() : multi_gather_attr<3>();
  if (at != BVC_OK) return at;
  if (b->dim == 2)
    k_gather_multi<2><<<grid, kMThreads, kMSum64, s>>>(pts, b->m_total, cache->packed, b->n_total, cache->k, u,
                                                       b->table, b->count, b->n_total, nullptr, 0);
  else
    k_gather_multi<3><<<grid, kMThreads, kMSum64, s>>>(pts, b->m_total, cache->packed, b->n_total, cache->k, u,
                                                       b->table, b->count, b->n_total, nullptr, 0);
  BVC_LAUNCH_CHECK();
  return BVC_OK;
}
extern "C" bvc_status bvc_batch_evaluate(bvc_batch b, const bvc_multi_cache* cache, const float* pts, double* u,
                                         bvc_stream stream) {
  return bvc::note_status(bvc_batch_evaluate_impl(b, cache, pts, u, stream));
}

static bvc_status bvc_evaluate_adjoint_workspace_size_impl(int64_t m, size_t* bytes) {
  if (m < 0 || bytes == nullptr) return BVC_ERR_INVALID_ARG;
  *bytes = 256 + (size_t)m * 16;
  return BVC_OK;
}
extern "C" bvc_status bvc_evaluate_adjoint_workspace_size(int64_t m, size_t* bytes) {
  return bvc::note_status(bvc_evaluate_adjoint_workspace_size_impl(m, bytes));
}

static bvc_status bvc_evaluate_adjoint_impl(const bvc_cache* cache, const float* pts, int64_t m, const double* lam,
                                           double* adj_u, double* adj_q, double* adj_src, void* workspace,
                                           size_t workspace_bytes, bvc_stream stream) {
  if (cache == nullptr || (cache->dim != 2 && cache->dim != 3) || cache->n < 1 || cache->z == nullptr ||
      cache->nrm == nullptr || cache->jac == nullptr || adj_u == nullptr || adj_q == nullptr || m < 0 ||
      (m > 0 && (pts == nullptr || lam == nullptr || workspace == nullptr)))
    return BVC_ERR_INVALID_ARG;
  const bool src = adj_src != nullptr && cache->n_src_cand > 0;
  if (src && (cache->src_y == nullptr || cache->n_src_dev == nullptr)) return BVC_ERR_INVALID_ARG;
  if (cache->sigma != 0.0 || cache->clamp_c != 0.0) return BVC_ERR_UNSUPPORTED;  // the Poisson gather's transpose
  if (workspace_bytes < 256 + (size_t)m * 16) return BVC_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  const int D = cache->dim;
  if (m == 0) {
    BVC_CUDA_TRY(cudaMemsetAsync(adj_u, 0, (size_t)cache->n * 8, s));
    BVC_CUDA_TRY(cudaMemsetAsync(adj_q, 0, (size_t)cache->n * 8, s));
    if (src) BVC_CUDA_TRY(cudaMemsetAsync(adj_src, 0, (size_t)cache->n_src_cand * 8, s));
    return BVC_OK;
  }
  float4* pl = (float4*)workspace;
  {
    ProfScope ps("adjoint_pack", s);
    if (D == 2)
      k_pack_adj_pts<2><<<(unsigned)((m + 255) / 256), 256, 0, s>>>(pts, m, lam, pl);
    else
      k_pack_adj_pts<3><<<(unsigned)((m + 255) / 256), 256, 0, s>>>(pts, m, lam, pl);
    BVC_LAUNCH_CHECK();
  }
  const double N = (double)cache->n;
  const double ca = D == 2 ? cache->bnd_measure / 6.283185307179586476925 : cache->bnd_measure / 12.566370614359172953850;
  const double cb = D == 2 ? -ca * 0.34657359027997265471 : ca;
  {
    ProfScope ps("adjoint_gather_boundary", s);
    const unsigned grid = (unsigned)((cache->n + 256 * kAS - 1) / (256 * kAS));
    if (D == 2)
      k_gather_adj<2, false><<<grid, 256, 0, s>>>(pl, m, cache->z, cache->nrm, cache->jac, cache->n, nullptr, cache->n,
                                                  ca / N, cb / N, adj_u, adj_q);
    else
      k_gather_adj<3, false><<<grid, 256, 0, s>>>(pl, m, cache->z, cache->nrm, cache->jac, cache->n, nullptr, cache->n,
                                                  ca / N, cb / N, adj_u, adj_q);
    BVC_LAUNCH_CHECK();
  }
  if (src) {
    const int64_t nc = cache->n_src_cand;
    BVC_CUDA_TRY(cudaMemsetAsync(adj_src, 0, (size_t)nc * 8, s));
    // source term: u += (1/ncand) sum_j G(x, y_j) c_j, G = lg2(r^2) ln2/(4 pi) (2D), -1/(4 pi r) (3D)
    const double cs = D == 2 ? 0.34657359027997265471 / 6.283185307179586476925 : -1.0 / 12.566370614359172953850;
    ProfScope ps("adjoint_gather_source", s);
    const unsigned grid = (unsigned)((nc + 256 * kAS - 1) / (256 * kAS));
    if (D == 2)
      k_gather_adj<2, true><<<grid, 256, 0, s>>>(pl, m, cache->src_y, nullptr, nullptr, nc, cache->n_src_dev, nc,
                                                 cs / (double)nc, 0.0, adj_src, nullptr);
    else
      k_gather_adj<3, true><<<grid, 256, 0, s>>>(pl, m, cache->src_y, nullptr, nullptr, nc, cache->n_src_dev, nc,
                                                 cs / (double)nc, 0.0, adj_src, nullptr);
    BVC_LAUNCH_CHECK();
  }
  return BVC_OK;
}
extern "C" bvc_status bvc_evaluate_adjoint(const bvc_cache* cache, const float* pts, int64_t m, const double* lam,
                                           double* adj_u, double* adj_q, double* adj_src, void* workspace,
                                           size_t workspace_bytes, bvc_stream stream) {
  return bvc::note_status(bvc_evaluate_adjoint_impl(cache, pts, m, lam, adj_u, adj_q, adj_src, workspace, workspace_bytes, stream));
}
