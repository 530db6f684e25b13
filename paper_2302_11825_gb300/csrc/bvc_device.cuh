// bvc_device.cuh -- device building blocks shared by the library's kernels:
// Philox-4x32-10, problem-function evaluation, the canonical FP32
// closest-point distance and the BVH closest-point traversal.
//
// Canonical closest-point distance.  The primitive is stored as a (first
// vertex) and ab = b - a (and ac = c - a), each difference one FP32
// subtraction.  The squared distance from p is the following fixed sequence
// of correctly rounded FP32 operations (no contraction):
//   segment:  ap = p - a; num = fma(ap.y, ab.y, ap.x*ab.x);
//             den = fma(ab.y, ab.y, ab.x*ab.x); inv = 1/den (one FP32
//             division, precomputed per segment);
//             num <= 0:    d2 = fma(ap.y, ap.y, ap.x*ap.x)
//             num >= den:  bp = ap - ab; d2 = fma(bp.y, bp.y, bp.x*bp.x)
//             otherwise:   c = fma(ap.x, ab.y, -(ap.y*ab.x)); d2 = (c*c)*inv
//   triangle: the Voronoi-region classification of Ericson, "Real-Time
//             Collision Detection" Sec. 5.1.5, written on (ap, ab, ac) with
//             dot(u,v) = fma(u.z, v.z, fma(u.y, v.y, u.x*v.x)),
//             bp = ap - ab, cp = ap - ac and the difference vector p - closest
//             formed directly with fma (see tri_closest below).
// Ties in d2 go to the lowest primitive index.  The BVH prunes a box only
// when its distance exceeds sqrt(best) + tau (tau = 2^-18 x bbox diagonal,
// far above the rounding of the expressions above), so the traversal
// returns exactly the brute-force argmin of these FP32 numbers.
#pragma once

#include <cstdint>

#include "bvc_internal.h"

namespace bvc {

constexpr float kPiF = 3.14159265358979323846f;

// Debug builds (BVC_DEBUG=1) check the tree links, leaf ranges and
// traversal stack depth before every access; a failed check sets the
// geometry's status flag kFlagBounds (bvc_geometry_stats returns
// BVC_ERR_BOUNDS), skips the access and lets the query finish.  Release
// builds compile the checks out.
#ifndef BVC_DEBUG
#define BVC_DEBUG 0
#endif
constexpr int kTravStack = 24;  // traversal stack entries; the BVH builder bounds the depth by 24
__device__ __forceinline__ bool dbg_bad_at(unsigned long long* stats, bool bad) {
  if (BVC_DEBUG && bad) {
    atomicOr(&stats[kStatFlags], kFlagBounds);
    return true;
  }
  return false;
}
__device__ __forceinline__ bool dbg_bad(const DevGeometry& G, bool bad) { return dbg_bad_at(G.stats, bad); }

// ----------------------------------------------------------------- Philox
// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): per round two 32x32
// multiplies by the round constants, xor of the high halves with the other
// counter words and the key, and a Weyl bump of the key between rounds.
struct U4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                            uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  return U4{c0, c1, c2, c3};
}

__device__ __forceinline__ U4 philox_draw(uint64_t seed, uint64_t id, uint32_t word2, uint32_t tag) {
  return philox4x32_10((uint32_t)id, (uint32_t)(id >> 32), word2, tag, (uint32_t)seed, (uint32_t)(seed >> 32));
}

// Uniform in (0,1): odd multiples of 2^-24, exact in FP32 and FP64.
__device__ __forceinline__ float u01f(uint32_t r) { return (float)((r >> 9) * 2u + 1u) * 0x1p-24f; }
__device__ __forceinline__ double u01d(uint32_t r) { return (double)((r >> 9) * 2u + 1u) * 0x1p-24; }

// ------------------------------------------------------- problem functions
// FAST: exp via the SFU (__expf, a few ulp), for the walks; the accurate
// expf elsewhere.
template <int D, bool FAST = false>
__device__ __forceinline__ float ex(float v) {
  return FAST ? __expf(v) : expf(v);
}

template <int D, bool FAST = false>
__device__ __forceinline__ float eval_fn(const DevFunction& fn, const float* x) {
  float v = 0.0f;
  for (int t = 0; t < fn.n_terms; ++t) {
    const float* c = fn.c + fn.off[t];
    const int nc = fn.nc[t];
    switch (fn.kind[t]) {
      case BVC_FN_POLY: {
        float xp[5], yp[5], zp[5];
        xp[0] = yp[0] = zp[0] = 1.0f;
#pragma unroll
        for (int e = 1; e < 5; ++e) {
          xp[e] = xp[e - 1] * x[0];
          yp[e] = yp[e - 1] * x[1];
          zp[e] = D == 3 ? zp[e - 1] * x[D == 3 ? 2 : 0] : 0.0f;
        }
        int idx = 0;
        for (int tt = 0; tt <= 4 && idx < nc; ++tt) {
          if (D == 2) {
            for (int i = tt; i >= 0 && idx < nc; --i, ++idx) v = fmaf(c[idx], xp[i] * yp[tt - i], v);
          } else {
            for (int i = tt; i >= 0 && idx < nc; --i)
              for (int j = tt - i; j >= 0 && idx < nc; --j, ++idx) v = fmaf(c[idx], xp[i] * yp[j] * zp[tt - i - j], v);
          }
        }
        break;
      }
      case BVC_FN_GAUSS: {  // device layout: [-1/(2s^2), (A, c[D])...]
        const float neg = c[0];
        for (int k = 1; k + D < nc; k += 1 + D) {
          float r2 = 0.0f;
#pragma unroll
          for (int a = 0; a < D; ++a) {
            const float d = x[a] - c[k + 1 + a];
            r2 = fmaf(d, d, r2);
          }
          v = fmaf(c[k], ex<D, FAST>(r2 * neg), v);
        }
        break;
      }
      case BVC_FN_GAUSS_LAPLACIAN: {  // device layout: [-1/(2s^2), 1/s^4, -D/s^2, (A, c[D])...]
        const float neg = c[0], q4 = c[1], qd = c[2];
        for (int k = 3; k + D < nc; k += 1 + D) {
          float r2 = 0.0f;
#pragma unroll
          for (int a = 0; a < D; ++a) {
            const float d = x[a] - c[k + 1 + a];
            r2 = fmaf(d, d, r2);
          }
          v = fmaf(c[k] * fmaf(r2, q4, qd), ex<D, FAST>(r2 * neg), v);
        }
        break;
      }
      case BVC_FN_EXP_TRIG:
        if (D == 3) v = fmaf(c[0] * ex<D, FAST>(c[1] * x[D == 3 ? 2 : 0]), cosf(c[2] * x[0]) * sinf(c[3] * x[1]), v);
        break;
      case BVC_FN_EXP_COS:
        v = fmaf(c[0] * ex<D, FAST>(c[1] * x[D - 1]), cosf(c[2] * x[0]), v);
        break;
      default:
        break;
    }
  }
  return v;
}

// Gradient of a problem function (a mixed problem's Neumann data is
// h = n . grad(potential)); kinds as eval_fn.
template <int D>
__device__ __forceinline__ void eval_fn_grad(const DevFunction& fn, const float* x, float* g) {
#pragma unroll
  for (int a = 0; a < D; ++a) g[a] = 0.0f;
  for (int t = 0; t < fn.n_terms; ++t) {
    const float* c = fn.c + fn.off[t];
    const int nc = fn.nc[t];
    switch (fn.kind[t]) {
      case BVC_FN_POLY: {
        // powers p[e] = x^e and derivatives dp[e] = e x^(e-1) per axis
        float xp[3][5], dp[3][5];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const float v = a < D ? x[a < D ? a : 0] : 0.0f;
          xp[a][0] = 1.0f;
          dp[a][0] = 0.0f;
#pragma unroll
          for (int e = 1; e < 5; ++e) {
            dp[a][e] = (float)e * xp[a][e - 1];
            xp[a][e] = xp[a][e - 1] * v;
          }
        }
        int idx = 0;
        for (int tt = 0; tt <= 4 && idx < nc; ++tt) {
          if (D == 2) {
            for (int i = tt; i >= 0 && idx < nc; --i, ++idx) {
              const int j = tt - i;
              g[0] = fmaf(c[idx], dp[0][i] * xp[1][j], g[0]);
              g[1] = fmaf(c[idx], xp[0][i] * dp[1][j], g[1]);
            }
          } else {
            for (int i = tt; i >= 0 && idx < nc; --i)
              for (int j = tt - i; j >= 0 && idx < nc; --j, ++idx) {
                const int k = tt - i - j;
                g[0] = fmaf(c[idx], dp[0][i] * xp[1][j] * xp[2][k], g[0]);
                g[1] = fmaf(c[idx], xp[0][i] * dp[1][j] * xp[2][k], g[1]);
                g[D - 1] = fmaf(c[idx], xp[0][i] * xp[1][j] * dp[2][k], g[D - 1]);
              }
          }
        }
        break;
      }
      case BVC_FN_GAUSS:
      case BVC_FN_GAUSS_LAPLACIAN: {
        // GAUSS: A e, e = exp(neg r2), grad = 2 neg A e d (d = x - centre);
        // GAUSS_LAPLACIAN: A q e, q = r2 q4 + qd, grad = A e d (2 q4 + 2 neg q)
        const bool lap = fn.kind[t] == BVC_FN_GAUSS_LAPLACIAN;
        const float neg = c[0], q4 = lap ? c[1] : 0.0f, qd = lap ? c[2] : 0.0f;
        for (int k = lap ? 3 : 1; k + D < nc; k += 1 + D) {
          float d[D], r2 = 0.0f;
#pragma unroll
          for (int a = 0; a < D; ++a) {
            d[a] = x[a] - c[k + 1 + a];
            r2 = fmaf(d[a], d[a], r2);
          }
          const float e = c[k] * expf(r2 * neg);
          const float fac = lap ? e * (2.0f * q4 + 2.0f * neg * fmaf(r2, q4, qd)) : 2.0f * neg * e;
#pragma unroll
          for (int a = 0; a < D; ++a) g[a] = fmaf(fac, d[a], g[a]);
        }
        break;
      }
      case BVC_FN_EXP_TRIG:
        if (D == 3) {
          const float e = c[0] * expf(c[1] * x[D == 3 ? 2 : 0]);
          const float cx = cosf(c[2] * x[0]), sx = sinf(c[2] * x[0]);
          const float cy = cosf(c[3] * x[1]), sy = sinf(c[3] * x[1]);
          g[0] = fmaf(-c[2] * e * sx, sy, g[0]);
          g[1] = fmaf(c[3] * e * cx, cy, g[1]);
          g[D - 1] = fmaf(c[1] * e * cx, sy, g[D - 1]);
        }
        break;
      case BVC_FN_EXP_COS: {
        const float e = c[0] * expf(c[1] * x[D - 1]);
        g[0] = fmaf(-c[2] * e, sinf(c[2] * x[0]), g[0]);
        g[D - 1] = fmaf(c[1] * e, cosf(c[2] * x[0]), g[D - 1]);
        break;
      }
      default:
        break;
    }
  }
}

// Boundary data from vertex values (the differentiable parameterisation of
// g): at a point p of element e (caller numbering), g is the linear
// interpolation of the element's vertex values -- segment: projection
// parameter t = (p-a).(b-a)/|b-a|^2 clamped to [0,1]; triangle: barycentric
// coordinates of p.  Returns the vertex ids and their weights.
template <int D>
__device__ __forceinline__ void vertex_weights(const DevGeometry& G, int32_t e, const float* p, int32_t* vid,
                                               float* w) {
  if (dbg_bad(G, e < 0 || e >= G.n_prims)) {
#pragma unroll
    for (int a = 0; a < D; ++a) vid[a] = 0, w[a] = 0.0f;
    return;
  }
#pragma unroll
  for (int a = 0; a < D; ++a) vid[a] = __ldg(&G.idx[(int64_t)e * D + a]);
  if (D == 2) {
    const float ax = __ldg(&G.verts[2 * (int64_t)vid[0]]), ay = __ldg(&G.verts[2 * (int64_t)vid[0] + 1]);
    const float abx = __ldg(&G.verts[2 * (int64_t)vid[1]]) - ax, aby = __ldg(&G.verts[2 * (int64_t)vid[1] + 1]) - ay;
    float t = fmaf(p[1] - ay, aby, (p[0] - ax) * abx) / fmaf(aby, aby, abx * abx);
    t = fminf(fmaxf(t, 0.0f), 1.0f);
    w[0] = 1.0f - t;
    w[D - 1] = t;
  } else {
    float v0[3], v1[3], v2[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float o = __ldg(&G.verts[3 * (int64_t)vid[0] + a]);
      v0[a] = __ldg(&G.verts[3 * (int64_t)vid[1 % D] + a]) - o;
      v1[a] = __ldg(&G.verts[3 * (int64_t)vid[2 % D] + a]) - o;
      v2[a] = p[a % D] - o;
    }
    const float d00 = fmaf(v0[2], v0[2], fmaf(v0[1], v0[1], v0[0] * v0[0]));
    const float d01 = fmaf(v0[2], v1[2], fmaf(v0[1], v1[1], v0[0] * v1[0]));
    const float d11 = fmaf(v1[2], v1[2], fmaf(v1[1], v1[1], v1[0] * v1[0]));
    const float d20 = fmaf(v2[2], v0[2], fmaf(v2[1], v0[1], v2[0] * v0[0]));
    const float d21 = fmaf(v2[2], v1[2], fmaf(v2[1], v1[1], v2[0] * v1[0]));
    const float inv = 1.0f / fmaf(d00, d11, -d01 * d01);
    const float bv = fmaf(d11, d20, -d01 * d21) * inv, bw = fmaf(d00, d21, -d01 * d20) * inv;
    w[0] = 1.0f - bv - bw;
    w[1 % D] = bv;
    w[2 % D] = bw;
  }
}

template <int D>
__device__ __forceinline__ float vertex_g(const DevGeometry& G, const float* __restrict__ gv, int32_t e,
                                          const float* p) {
  int32_t vid[D];
  float w[D];
  vertex_weights<D>(G, e, p, vid, w);
  float v = 0.0f;
#pragma unroll
  for (int a = 0; a < D; ++a) v = fmaf(w[a], __ldg(&gv[vid[a]]), v);
  return v;
}

// Shape functions of the bumps of a one-term GAUSS or GAUSS_LAPLACIAN
// source (f = sum_k A_k psi_k): psi_k(y) for k < kMaxBumps.
constexpr int kMaxBumps = 8;
template <int D>
__device__ __forceinline__ void bump_shapes(const DevFunction& fn, const float* y, float* psi) {
  const float* c = fn.c + fn.off[0];
  const bool lap = fn.kind[0] == BVC_FN_GAUSS_LAPLACIAN;
  const int head = lap ? 3 : 1;
  const float neg = c[0], q4 = lap ? c[1] : 0.0f, qd = lap ? c[2] : 0.0f;
#pragma unroll
  for (int k = 0; k < kMaxBumps; ++k) {
    const int o = head + k * (1 + D);
    float v = 0.0f;
    if (o + D < fn.nc[0]) {
      float r2 = 0.0f;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const float d = y[a] - c[o + 1 + a];
        r2 = fmaf(d, d, r2);
      }
      v = __expf(r2 * neg);
      if (lap) v *= fmaf(r2, q4, qd);
    }
    psi[k] = v;
  }
}

// ------------------------------------------- screened Poisson (sigma > 0)
// Modified Bessel functions in FP32 by the polynomial approximations of
// Abramowitz and Stegun, Handbook of Mathematical Functions, 9.8.1-9.8.8
// (absolute or relative error below 2.2e-7).  The large-argument forms are
// returned with their exponential factored out, so that the walk's factors
// and the gather's kernels never overflow:
//   i0s(t) = sqrt(t) e^-t I0(t), i1s(t) = sqrt(t) e^-t I1(t)  (t >= 3.75)
//   k0s(t) = sqrt(t) e^t K0(t),  k1s(t) = sqrt(t) e^t K1(t)   (t >= 2)
__device__ __forceinline__ float bessel_i0_small(float t) {  // 9.8.1, |t| <= 3.75
  const float y = (t / 3.75f) * (t / 3.75f);
  return fmaf(y, fmaf(y, fmaf(y, fmaf(y, fmaf(y, fmaf(y, 0.0045813f, 0.0360768f), 0.2659732f), 1.2067492f),
                                   3.0899424f), 3.5156229f), 1.0f);
}
__device__ __forceinline__ float bessel_i0s_large(float t) {  // 9.8.2, t >= 3.75
  const float y = 3.75f / t;
  return fmaf(y, fmaf(y, fmaf(y, fmaf(y, fmaf(y, fmaf(y, fmaf(y, fmaf(y, 0.00392377f, -0.01647633f), 0.02635537f),
                                                                -0.02057706f), 0.00916281f), -0.00157565f),
                                   0.00225319f), 0.01328592f), 0.39894228f);
}
__device__ __forceinline__ float bessel_i1_small(float t) {  // 9.8.3, |t| <= 3.75
  const float y = (t / 3.75f) * (t / 3.75f);
  return t * fmaf(y, fmaf(y, fmaf(y, fmaf(y, fmaf(y, fmaf(y, 0.00032411f, 0.00301532f), 0.02658733f), 0.15084934f),
                                       0.51498869f), 0.87890594f), 0.5f);
}
__device__ __forceinline__ float bessel_i1s_large(float t) {  // 9.8.4, t >= 3.75
  const float y = 3.75f / t;
  return fmaf(y, fmaf(y, fmaf(y, fmaf(y, fmaf(y, fmaf(y, fmaf(y, fmaf(y, -0.00420059f, 0.01787654f), -0.02895312f),
                                                                0.02282967f), -0.01031555f), 0.00163801f),
                                   -0.00362018f), -0.03988024f), 0.39894228f);
}
// K0, K1 for t <= 2 (9.8.5, 9.8.7) and the scaled forms for t >= 2 (9.8.6, 9.8.8).
__device__ __forceinline__ float bessel_k0_small(float t) {
  const float y = 0.25f * t * t;
  const float p = fmaf(y, fmaf(y, fmaf(y, fmaf(y, fmaf(y, fmaf(y, 0.0000074f, 0.0001075f), 0.00262698f), 0.0348859f),
                                       0.23069756f), 0.4227842f), -0.57721566f);
  return fmaf(-__logf(0.5f * t), bessel_i0_small(t), p);
}
__device__ __forceinline__ float bessel_k0s_large(float t) {
  const float y = 2.0f / t;
  return fmaf(y, fmaf(y, fmaf(y, fmaf(y, fmaf(y, fmaf(y, 0.00053208f, -0.0025154f), 0.00587872f), -0.01062446f),
                                   0.02189568f), -0.07832358f), 1.25331414f);
}
__device__ __forceinline__ float bessel_k1_small(float t) {  // returns K1(t)
  const float y = 0.25f * t * t;
  const float p = fmaf(y, fmaf(y, fmaf(y, fmaf(y, fmaf(y, fmaf(y, -0.00004686f, -0.00110404f), -0.01919402f),
                                                 -0.18156897f), -0.67278579f), 0.15443144f), 1.0f);
  return fmaf(__logf(0.5f * t), bessel_i1_small(t), p / t);
}
__device__ __forceinline__ float bessel_k1s_large(float t) {
  const float y = 2.0f / t;
  return fmaf(y, fmaf(y, fmaf(y, fmaf(y, fmaf(y, fmaf(y, -0.00068245f, 0.00325614f), -0.00780353f), 0.01504268f),
                                   -0.0365562f), 0.23498619f), 1.25331414f);
}

// The walk's ball factors (t = R sqrt(sigma)): u(centre) = C avg_sphere u and
// grad u(centre) = (D/R) Qg avg_sphere[u nu]:
//   3D  C = t / sinh t,   Qg = t^3 / (3 (t cosh t - sinh t))   (series below 0.5)
//   2D  C = 1 / I0(t),    Qg = t / (2 I1(t))
template <int D>
__device__ __forceinline__ void screened_factors(float t, float& C, float& Qg) {
  if (D == 3) {
    if (t < 0.5f) {
      const float t2 = t * t;
      C = 1.0f / fmaf(t2, fmaf(t2, fmaf(t2, 1.0f / 5040.0f, 1.0f / 120.0f), 1.0f / 6.0f), 1.0f);
      Qg = 1.0f / fmaf(t2, fmaf(t2, fmaf(t2, 1.0f / 1330560.0f * t2 + 1.0f / 15120.0f, 1.0f / 280.0f), 1.0f / 10.0f),
                       1.0f);
    } else {
      const float e = __expf(-t);            // sinh t = (1 - e^-2t) e^t / 2
      const float e2 = e * e;
      const float sh = 0.5f * (1.0f - e2), ch = 0.5f * (1.0f + e2);  // times e^t
      C = t * 2.0f * e / (1.0f - e2);
      Qg = t * t * t * e / (3.0f * fmaf(t, ch, -sh));
    }
  } else {
    if (t <= 3.75f) {
      C = 1.0f / bessel_i0_small(t);
      Qg = t / (2.0f * bessel_i1_small(t));
    } else {
      const float sq = sqrtf(t) * __expf(-t);
      C = sq / bessel_i0s_large(t);
      Qg = t * sq / (2.0f * bessel_i1s_large(t));
    }
  }
}

// Exponentially scaled forms for all t > 0, so that ratios of large
// arguments never overflow: e^t K0(t), e^t K1(t), e^-t I0(t), e^-t I1(t).
__device__ __forceinline__ float bessel_k0e(float t) {
  return t <= 2.0f ? bessel_k0_small(t) * __expf(t) : bessel_k0s_large(t) * rsqrtf(t);
}
__device__ __forceinline__ float bessel_k1e(float t) {
  return t <= 2.0f ? bessel_k1_small(t) * __expf(t) : bessel_k1s_large(t) * rsqrtf(t);
}
__device__ __forceinline__ float bessel_i0e(float t) {
  return t <= 3.75f ? bessel_i0_small(t) * __expf(-t) : bessel_i0s_large(t) * rsqrtf(t);
}
__device__ __forceinline__ float bessel_i1e(float t) {
  return t <= 3.75f ? bessel_i1_small(t) * __expf(-t) : bessel_i1s_large(t) * rsqrtf(t);
}
// e^-t (t cosh t - sinh t): the series t^3/3 (1 + t^2/10 + t^4/280 + t^6/15120)
// below 0.5, else ((t - 1) + e^-2t (t + 1)) / 2.
__device__ __forceinline__ float jcosh_e(float t) {
  if (t < 0.5f) {
    const float t2 = t * t;
    return __expf(-t) * (t * t2 * (1.0f / 3.0f)) *
           fmaf(t2, fmaf(t2, fmaf(t2, 1.0f / 15120.0f, 1.0f / 280.0f), 0.1f), 1.0f);
  }
  return 0.5f * fmaf(__expf(-2.0f * t), t + 1.0f, t - 1.0f);
}

// Source weights of one screened step ((Delta - sigma) u = f, k = sqrt(sigma)):
// the ball B(x, R) gives u(x) = C avg_sphere u - int_B G f, G the Green's
// function of (sigma - Delta) on the ball (zero on its sphere) seen from the
// centre, and the centre gradient of the source integral int_B w phi f, phi
// the l = 1 radial mode that vanishes at R:
//   2D  G = [K0(kr) - K0(kR) I0(kr)/I0(kR)] / (2 pi)
//       phi = k [K1(kr) - K1(kR) I1(kr)/I1(kR)] / (2 pi)
//   3D  G = sinh(k (R - r)) / (4 pi r sinh kR)
//       phi = [Q(r) - Q(R) J(kr)/J(kR)] / (4 pi r^2),  Q(r) = e^-kr (kr + 1), J(t) = t cosh t - sinh t.
// With the step's sample at radius rho (density 1 / (R |S| rho^(D-1))):
// wu = -|S| R rho^(D-1) G(rho) and wg = -|S| R rho^(D-1) phi(rho) -- at k ->
// 0 the Poisson weights -R rho ln(R/rho), -rho (R - rho) and -R (1 - (rho/R)^D).
template <int D>
__device__ __forceinline__ void screened_step_weights(float k, float R, float rho, bool want_g, float& wu,
                                                      float& wg) {
  const float tr = k * rho, tR = k * R;
  if (D == 2) {
    const float er = __expf(-tr), cross = __expf(tr - 2.0f * tR);
    const float G = fmaf(-cross * bessel_k0e(tR), bessel_i0e(tr) / bessel_i0e(tR), er * bessel_k0e(tr));
    wu = -R * rho * G;
    if (want_g) {
      const float phi = fmaf(-cross * bessel_k1e(tR), bessel_i1e(tr) / bessel_i1e(tR), er * bessel_k1e(tr));
      wg = -R * tr * phi;
    }
  } else {
    // sinh(tR - tr) / sinh(tR) = e^-tr (1 - e^-2(tR - tr)) / (1 - e^-2tR)
    wu = -R * rho * __expf(-tr) * (expm1f(-2.0f * (tR - tr)) / expm1f(-2.0f * tR));
    if (want_g)
      wg = -R * fmaf(-(tR + 1.0f) * __expf(tr - 2.0f * tR), jcosh_e(tr) / jcosh_e(tR), __expf(-tr) * (tr + 1.0f));
  }
}

// Screened walk on stars (Sec. 3.1 with sigma > 0).  The ball's Green's
// function G of (sigma - Delta) on B(x, R), zero on its sphere (see
// screened_step_weights), at distance rho from the centre:
//   2D  [K0(k rho) - K0(kR) I0(k rho)/I0(kR)] / (2 pi)
//   3D  sinh(k (R - rho)) / (4 pi rho sinh kR)
template <int D>
__device__ __forceinline__ float ball_green_sigma(float k, float R, float rho) {
  const float tr = k * rho, tR = k * R;
  if (D == 2) {
    const float G = fmaf(-__expf(tr - 2.0f * tR) * bessel_k0e(tR), bessel_i0e(tr) / bessel_i0e(tR),
                         __expf(-tr) * bessel_k0e(tr));
    return G * (0.5f / kPiF);
  }
  return __expf(-tr) * (expm1f(-2.0f * (tR - tr)) / expm1f(-2.0f * tR)) * (0.25f / kPiF) / rho;
}
// The factor a step's direction carries to the first boundary point it
// meets at distance r <= R: W(r) = -|S| r^(D-1) dG/dr (Green's identity on
// the star-shaped region with the ball's G; W(R) is the ball's mean-value
// factor, W -> 1 as r -> 0):
//   2D  kr [K1(kr) + K0(kR) I1(kr)/I0(kR)]
//   3D  [kr cosh(k (R - r)) + sinh(k (R - r))] / sinh kR
template <int D>
__device__ __forceinline__ float star_kernel_sigma(float k, float R, float r) {
  const float tr = k * r, tR = k * R;
  if (!(tr > 0.0f)) return 1.0f;
  if (D == 2)
    return tr * fmaf(__expf(tr - 2.0f * tR) * bessel_k0e(tR), bessel_i1e(tr) / bessel_i0e(tR),
                     __expf(-tr) * bessel_k1e(tr));
  const float ea = expm1f(-2.0f * (tR - tr));  // e^-2(tR - tr) - 1
  return __expf(-tr) * fmaf(tr, 2.0f + ea, -ea) / -expm1f(-2.0f * tR);
}

// ------------------------------------------- canonical closest-point distance
// S = (a.x, a.y, ab.x, ab.y), inv = 1/|ab|^2.
__device__ __forceinline__ float seg_d2(const float4 S, float inv, float px, float py) {
  const float apx = __fsub_rn(px, S.x), apy = __fsub_rn(py, S.y);
  const float num = __fmaf_rn(apy, S.w, __fmul_rn(apx, S.z));
  const float den = __fmaf_rn(S.w, S.w, __fmul_rn(S.z, S.z));
  const float bx = __fsub_rn(apx, S.z), by = __fsub_rn(apy, S.w);
  const float c = __fmaf_rn(apx, S.w, -__fmul_rn(apy, S.z));
  const float da = __fmaf_rn(apy, apy, __fmul_rn(apx, apx));
  const float db = __fmaf_rn(by, by, __fmul_rn(bx, bx));
  const float dc = __fmul_rn(__fmul_rn(c, c), inv);
  return num <= 0.0f ? da : (num >= den ? db : dc);
}

// p - (closest point on the segment), for the winning segment of a query.
__device__ __forceinline__ void seg_diff(const float4 S, float inv, float px, float py, float& dx, float& dy) {
  const float apx = __fsub_rn(px, S.x), apy = __fsub_rn(py, S.y);
  const float num = __fmaf_rn(apy, S.w, __fmul_rn(apx, S.z));
  const float den = __fmaf_rn(S.w, S.w, __fmul_rn(S.z, S.z));
  const float t = num <= 0.0f ? 0.0f : (num >= den ? 1.0f : __fmul_rn(num, inv));
  dx = __fmaf_rn(-t, S.z, apx);
  dy = __fmaf_rn(-t, S.w, apy);
}

__device__ __forceinline__ float dot3c(float ux, float uy, float uz, float vx, float vy, float vz) {
  return __fmaf_rn(uz, vz, __fmaf_rn(uy, vy, __fmul_rn(ux, vx)));
}

// Returns d2 and the difference vector df = p - closest point.
__device__ __forceinline__ float tri_closest(const float4 A, const float4 B, const float4 Cc, const float* p,
                                             float* df) {
  const float apx = __fsub_rn(p[0], A.x), apy = __fsub_rn(p[1], A.y), apz = __fsub_rn(p[2], A.z);
  const float abx = B.x, aby = B.y, abz = B.z, acx = Cc.x, acy = Cc.y, acz = Cc.z;
  const float d1 = dot3c(abx, aby, abz, apx, apy, apz), d2 = dot3c(acx, acy, acz, apx, apy, apz);
  if (d1 <= 0.0f && d2 <= 0.0f) {
    df[0] = apx;
    df[1] = apy;
    df[2] = apz;
    return dot3c(apx, apy, apz, apx, apy, apz);
  }
  const float bpx = __fsub_rn(apx, abx), bpy = __fsub_rn(apy, aby), bpz = __fsub_rn(apz, abz);
  const float d3 = dot3c(abx, aby, abz, bpx, bpy, bpz), d4 = dot3c(acx, acy, acz, bpx, bpy, bpz);
  if (d3 >= 0.0f && d4 <= d3) {
    df[0] = bpx;
    df[1] = bpy;
    df[2] = bpz;
    return dot3c(bpx, bpy, bpz, bpx, bpy, bpz);
  }
  const float vc = __fmaf_rn(d1, d4, -__fmul_rn(d3, d2));
  if (vc <= 0.0f && d1 >= 0.0f && d3 <= 0.0f) {
    const float v = __fdiv_rn(d1, __fsub_rn(d1, d3));
    df[0] = __fmaf_rn(-v, abx, apx);
    df[1] = __fmaf_rn(-v, aby, apy);
    df[2] = __fmaf_rn(-v, abz, apz);
    return dot3c(df[0], df[1], df[2], df[0], df[1], df[2]);
  }
  const float cpx = __fsub_rn(apx, acx), cpy = __fsub_rn(apy, acy), cpz = __fsub_rn(apz, acz);
  const float d5 = dot3c(abx, aby, abz, cpx, cpy, cpz), d6 = dot3c(acx, acy, acz, cpx, cpy, cpz);
  if (d6 >= 0.0f && d5 <= d6) {
    df[0] = cpx;
    df[1] = cpy;
    df[2] = cpz;
    return dot3c(cpx, cpy, cpz, cpx, cpy, cpz);
  }
  const float vb = __fmaf_rn(d5, d2, -__fmul_rn(d1, d6));
  if (vb <= 0.0f && d2 >= 0.0f && d6 <= 0.0f) {
    const float w = __fdiv_rn(d2, __fsub_rn(d2, d6));
    df[0] = __fmaf_rn(-w, acx, apx);
    df[1] = __fmaf_rn(-w, acy, apy);
    df[2] = __fmaf_rn(-w, acz, apz);
    return dot3c(df[0], df[1], df[2], df[0], df[1], df[2]);
  }
  const float va = __fmaf_rn(d3, d6, -__fmul_rn(d5, d4));
  const float e43 = __fsub_rn(d4, d3), e56 = __fsub_rn(d5, d6);
  if (va <= 0.0f && e43 >= 0.0f && e56 >= 0.0f) {
    const float w = __fdiv_rn(e43, __fadd_rn(e43, e56));
    df[0] = __fmaf_rn(-w, __fsub_rn(acx, abx), bpx);
    df[1] = __fmaf_rn(-w, __fsub_rn(acy, aby), bpy);
    df[2] = __fmaf_rn(-w, __fsub_rn(acz, abz), bpz);
    return dot3c(df[0], df[1], df[2], df[0], df[1], df[2]);
  }
  const float denom = __frcp_rn(__fadd_rn(__fadd_rn(va, vb), vc));
  const float v = __fmul_rn(vb, denom), w = __fmul_rn(vc, denom);
  df[0] = __fmaf_rn(-w, acx, __fmaf_rn(-v, abx, apx));
  df[1] = __fmaf_rn(-w, acy, __fmaf_rn(-v, aby, apy));
  df[2] = __fmaf_rn(-w, acz, __fmaf_rn(-v, abz, apz));
  return dot3c(df[0], df[1], df[2], df[0], df[1], df[2]);
}

// ------------------------------------------------------- BVH traversal
template <int D>
struct Hit {
  float d2;
  int32_t id;   // caller's element index
  int32_t q;    // BVH-order record of the element
  float df[D];  // p - closest point (3D: kept during the query; 2D: by finish_hit)
};

__device__ __forceinline__ float box_d2_2(float lox, float loy, float hix, float hiy, const float* p) {
  const float dx = fmaxf(fmaxf(lox - p[0], p[0] - hix), 0.0f);
  const float dy = fmaxf(fmaxf(loy - p[1], p[1] - hiy), 0.0f);
  return fmaf(dy, dy, dx * dx);
}

__device__ __forceinline__ float box_d2_3(float lox, float loy, float loz, float hix, float hiy, float hiz,
                                          const float* p) {
  const float dx = fmaxf(fmaxf(lox - p[0], p[0] - hix), 0.0f);
  const float dy = fmaxf(fmaxf(loy - p[1], p[1] - hiy), 0.0f);
  const float dz = fmaxf(fmaxf(loz - p[2], p[2] - hiz), 0.0f);
  return fmaf(dz, dz, fmaf(dy, dy, dx * dx));
}

// Squared distance from p to the slab dmin <= n . x <= dmax (an unbounded
// slab has n = 0 and gives 0).
template <int D>
__device__ __forceinline__ float slab_d2(float nx, float ny, float nz, float dmin, float dmax, const float* p) {
  const float s = D == 2 ? fmaf(ny, p[1], nx * p[0]) : fmaf(nz, p[D - 1], fmaf(ny, p[1], nx * p[0]));
  const float d = fmaxf(fmaxf(s - dmax, dmin - s), 0.0f);
  return d * d;
}

// One node fetch: the children's links and lower bounds on the squared
// distance from p to the elements below each child, max(box distance^2,
// slab distance^2) (the slab of a smooth patch is much thinner than its
// box).  Box distances are exact FP32 bounds; the slab distance's rounding
// (a few ulp of |p|) is far below the traversal's slack tau, which the
// pruning threshold already includes.
template <int D>
__device__ __forceinline__ void node_bounds(const DevGeometry& G, int node, const float* p, float& dl, float& dr,
                                            int32_t& cl, int32_t& cr) {
  if (dbg_bad(G, node < 0 || node >= G.n_nodes)) {  // both children out of reach
    dl = dr = __int_as_float(0x7f800000);
    cl = cr = ~0;
    return;
  }
  if (D == 2) {
    const float4 L = __ldg(&G.nodes[3 * node]), R = __ldg(&G.nodes[3 * node + 1]);
    const float4 C = __ldg(&G.nodes[3 * node + 2]);
    const float4 SL = __ldg(&G.slabs[2 * node]), SR = __ldg(&G.slabs[2 * node + 1]);
    dl = fmaxf(box_d2_2(L.x, L.y, L.z, L.w, p), slab_d2<2>(SL.x, SL.y, 0.0f, SL.z, SL.w, p));
    dr = fmaxf(box_d2_2(R.x, R.y, R.z, R.w, p), slab_d2<2>(SR.x, SR.y, 0.0f, SR.z, SR.w, p));
    cl = __float_as_int(C.x);
    cr = __float_as_int(C.y);
  } else {
    const float4 a = __ldg(&G.nodes[4 * node]), b = __ldg(&G.nodes[4 * node + 1]);
    const float4 c = __ldg(&G.nodes[4 * node + 2]), e = __ldg(&G.nodes[4 * node + 3]);
    const float4 s0 = __ldg(&G.slabs[3 * node]), s1 = __ldg(&G.slabs[3 * node + 1]);
    const float4 s2 = __ldg(&G.slabs[3 * node + 2]);
    dl = fmaxf(box_d2_3(a.x, a.y, a.z, a.w, b.x, b.y, p), slab_d2<3>(s0.x, s0.y, s0.z, s0.w, s1.x, p));
    dr = fmaxf(box_d2_3(b.z, b.w, c.x, c.y, c.z, c.w, p), slab_d2<3>(s1.y, s1.z, s1.w, s2.x, s2.y, p));
    cl = __float_as_int(e.x);
    cr = __float_as_int(e.y);
  }
}

// Work counters of the counting variant (node fetches, primitive tests).
struct TravCount {
  uint32_t nodes, prims;
};

template <int D, bool CNT>
__device__ __forceinline__ void test_leaf(const DevGeometry& G, int32_t enc, const float* p, Hit<D>& h, float& thr,
                                          TravCount& tc) {
  const int32_t e = ~enc;
  const int32_t first = e >> 4, count = e & 15;
  if (dbg_bad(G, first < 0 || (int64_t)first + count > G.n_prims)) return;
  if (CNT) tc.prims += (uint32_t)count;
  for (int32_t q = first; q < first + count; ++q) {
    if (D == 2) {
      const float4 S = __ldg(&G.prims[2 * q]), T = __ldg(&G.prims[2 * q + 1]);
      const float d2 = seg_d2(S, T.x, p[0], p[1]);
      const int32_t id = __float_as_int(T.y);
      if (d2 < h.d2 || (d2 == h.d2 && id < h.id)) {
        h.d2 = d2;
        h.id = id;
        h.q = q;
        const float sr = sqrtf(d2) + G.tau;
        thr = sr * sr;
      }
    } else {
      const float4 A = __ldg(&G.prims[3 * q]), B = __ldg(&G.prims[3 * q + 1]), Cc = __ldg(&G.prims[3 * q + 2]);
      float df[3];
      const float d2 = tri_closest(A, B, Cc, p, df);
      const int32_t id = __float_as_int(A.w);
      if (d2 < h.d2 || (d2 == h.d2 && id < h.id)) {
        h.d2 = d2;
        h.id = id;
        h.q = q;
#pragma unroll
        for (int a = 0; a < D; ++a) h.df[a] = df[D == 3 ? a : 0];
        const float sr = sqrtf(d2) + G.tau;
        thr = sr * sr;
      }
    }
  }
}

// Completes a hit: the difference vector p - closest point of the winner.
template <int D>
__device__ __forceinline__ void finish_hit(const DevGeometry& G, const float* p, Hit<D>& h) {
  if (D == 2 && h.q >= 0) {
    const float4 S = __ldg(&G.prims[2 * h.q]), T = __ldg(&G.prims[2 * h.q + 1]);
    seg_diff(S, T.x, p[0], p[1], h.df[0], h.df[D - 1]);
  }
}

// One node of the closest-primitive traversal: the children's bounds, leaf
// children tested, then the nearer child still within reach next (the
// farther one stacked when both are), else the nearest stacked node still
// within reach.  Returns true when the query is complete (call finish_hit).
// Stack in shared memory: stack[k * stride + lane_slot].
template <int D, bool CNT = false>
__device__ __forceinline__ bool closest_visit(const DevGeometry& G, const float* p, Hit<D>& h, float& thr,
                                              int& node, int& sp, int* snode, float* sdist, int stride,
                                              TravCount& tc) {
  int32_t cl, cr;
  float dl, dr;
  if (CNT) ++tc.nodes;
  node_bounds<D>(G, node, p, dl, dr, cl, cr);
  if (dr < dl) {
    const int32_t ti = cl;
    cl = cr;
    cr = ti;
    const float td = dl;
    dl = dr;
    dr = td;
  }
  bool tl = dl <= thr, tr = dr <= thr;
  if (tl && cl < 0) {
    test_leaf<D, CNT>(G, cl, p, h, thr, tc);
    tl = false;
    tr = dr <= thr;
  }
  if (tr && cr < 0) {
    test_leaf<D, CNT>(G, cr, p, h, thr, tc);
    tr = false;
  }
  if (tl && tr) {
    if (!dbg_bad(G, sp >= kTravStack)) {
      snode[sp * stride] = cr;
      sdist[sp * stride] = dr;
      ++sp;
    }
    node = cl;
    return false;
  }
  if (tl) {
    node = cl;
    return false;
  }
  if (tr) {
    node = cr;
    return false;
  }
  while (sp > 0) {
    --sp;
    if (sdist[sp * stride] <= thr) {
      node = snode[sp * stride];
      return false;
    }
  }
  return true;
}

// An empty hit: no primitive yet, infinite distance.
template <int D>
__device__ __forceinline__ void hit_reset(Hit<D>& h) {
  h.d2 = __int_as_float(0x7f800000);
  h.id = 0x7fffffff;
  h.q = -1;
#pragma unroll
  for (int a = 0; a < D; ++a) h.df[a] = 0.0f;
}

// Closest primitive to p.  Stack in shared memory: stack[k * stride + lane_slot].
template <int D, bool CNT = false>
__device__ __forceinline__ void bvh_closest(const DevGeometry& G, const float* p, Hit<D>& h, int* snode,
                                            float* sdist, int stride, TravCount& tc, int root = 0) {
  hit_reset<D>(h);
  float thr = __int_as_float(0x7f800000);
  int sp = 0;
  int node = root;
  while (!closest_visit<D, CNT>(G, p, h, thr, node, sp, snode, sdist, stride, tc)) {
  }
  finish_hit<D>(G, p, h);
}

}  // namespace bvc
