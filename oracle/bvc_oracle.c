/*
 * bvc_oracle.c -- plain, slow FP64 CPU oracle for Boundary Value Caching
 * (Miller, Sawhney, Crane, Gkioulekas, "Boundary Value Caching for Walk on
 * Spheres", SIGGRAPH 2023).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, header or constant table
 * with the CUDA library; the two meet only through the seeded inputs.
 *
 * Every routine follows the paper's definitions in the paper's order, in
 * double precision, with no blocking or fusion:
 *   - free-space Green's functions and derivatives ........ App. A, Eq. A1-A4
 *     (reading: G_3D = -1/(4 pi r), the sign implied by the printed
 *      gradient, normal derivative and second derivative)
 *   - boundary estimator, source estimator, gradients ..... Eq. 3-6, Alg. 1
 *   - walk on spheres with the ball Green's function ...... Sec. 3.1, Eq. 7
 *   - boundary sampling by a CDF over element measures .... Sec. 4 "Sampling"
 *   - offset Dirichlet boundary: the closed surface of the
 *     mesh with its vertices moved inward (reading below) ... Sec. 3.2
 *   - stratified uniform source samples ................... Sec. 4 "Sampling"
 * Randomness: Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11), written here from that definition.
 *
 * Decisions that pick an integer (closest primitive index, inside/outside
 * test of a candidate source point) have, besides the FP64 versions, a
 * "canonical FP32" form with a fixed operation order (explicit fmaf, no
 * contraction) so that the GPU path, which takes them in FP32, can be
 * checked bit-exactly.  This file must be compiled with -ffp-contract=off.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Philox-4x32-10 (SC'11).  Round: two 32x32->64 multiplies by the round     */
/* constants, a swap and xor with the key; the key is bumped by the Weyl     */
/* constants between rounds.                                                  */
/* ------------------------------------------------------------------------ */
static void philox_round(uint32_t c[4], const uint32_t k[2]) {
  const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
  const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
  const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
  const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
  const uint32_t n0 = hi1 ^ c[1] ^ k[0];
  const uint32_t n2 = hi0 ^ c[3] ^ k[1];
  c[0] = n0;
  c[1] = lo1;
  c[2] = n2;
  c[3] = lo0;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  uint32_t k[2] = {key[0], key[1]};
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k[0] += 0x9E3779B9u;
      k[1] += 0xBB67AE85u;
    }
    philox_round(c, k);
  }
  memcpy(out, c, sizeof(c));
}

/* Uniform in the open interval (0,1): odd multiples of 2^-24.  Every value is
 * exact in FP32 and FP64, so both sides of a parity test see the same number. */
double orc_u01(uint32_t r) { return ((double)(r >> 9) * 2.0 + 1.0) * 0x1p-24; }

/* One Philox draw for (id, word2, tag) under a 64-bit seed. */
static void draw(uint64_t seed, uint64_t id, uint32_t word2, uint32_t tag, double u[4]) {
  uint32_t ctr[4] = {(uint32_t)id, (uint32_t)(id >> 32), word2, tag};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t r[4];
  orc_philox4x32_10(ctr, key, r);
  for (int i = 0; i < 4; ++i) u[i] = orc_u01(r[i]);
}

/* ------------------------------------------------------------------------ */
/* Problem functions g and f (Eq. 1).  The paper passes them as callbacks;   */
/* here a function is a sum of terms from a few closed families, encoded as  */
/* a flat array: [n_terms, (kind, n_coeffs, coeffs...) x n_terms].           */
/*   kind 1 POLY: monomials x^i y^j (z^k), total degree <= 4, ordered by      */
/*          degree t = 0..4, then i = t..0, then (3D) j = t-i..0.             */
/*   kind 2 GAUSS: [s, A_1, c_1(dim), A_2, c_2, ...]:                         */
/*          sum A_k exp(-|x-c_k|^2 / (2 s^2)).                                */
/*   kind 3 GAUSS_LAPLACIAN: same coefficients, value = Laplacian of GAUSS:   */
/*          sum A_k (|x-c_k|^2/s^4 - dim/s^2) exp(-|x-c_k|^2/(2 s^2)).       */
/*   kind 4 EXP_TRIG (3D): [A, alpha, beta, gamma]:                           */
/*          A exp(alpha z) cos(beta x) sin(gamma y).                          */
/*   kind 5 EXP_COS: [A, alpha, beta]: A exp(alpha x_last) cos(beta x_0)      */
/*          (x_last = y in 2D, z in 3D); Laplacian = (alpha^2 - beta^2) value. */
/* ------------------------------------------------------------------------ */
static double ipow(double x, int e) {
  double r = 1.0;
  for (int i = 0; i < e; ++i) r *= x;
  return r;
}

static double poly_eval(int dim, const double* c, int nc, const double* x) {
  double s = 0.0;
  int idx = 0;
  for (int t = 0; t <= 4 && idx < nc; ++t) {
    if (dim == 2) {
      for (int i = t; i >= 0 && idx < nc; --i, ++idx) s += c[idx] * ipow(x[0], i) * ipow(x[1], t - i);
    } else {
      for (int i = t; i >= 0 && idx < nc; --i)
        for (int j = t - i; j >= 0 && idx < nc; --j, ++idx)
          s += c[idx] * ipow(x[0], i) * ipow(x[1], j) * ipow(x[2], t - i - j);
    }
  }
  return s;
}

static double gauss_eval(int dim, const double* c, int nc, const double* x, int laplacian) {
  const double s = c[0];
  const int per = 1 + dim;
  double v = 0.0;
  for (int k = 0; 1 + (k + 1) * per <= nc; ++k) {
    const double* b = c + 1 + k * per;
    double r2 = 0.0;
    for (int a = 0; a < dim; ++a) r2 += (x[a] - b[1 + a]) * (x[a] - b[1 + a]);
    const double e = exp(-r2 / (2.0 * s * s));
    v += laplacian ? b[0] * (r2 / (s * s * s * s) - dim / (s * s)) * e : b[0] * e;
  }
  return v;
}

double orc_fn_eval(const double* spec, int dim, const double* x) {
  const int nt = (int)spec[0];
  const double* p = spec + 1;
  double v = 0.0;
  for (int t = 0; t < nt; ++t) {
    const int kind = (int)p[0], nc = (int)p[1];
    const double* c = p + 2;
    switch (kind) {
      case 1: v += poly_eval(dim, c, nc, x); break;
      case 2: v += gauss_eval(dim, c, nc, x, 0); break;
      case 3: v += gauss_eval(dim, c, nc, x, 1); break;
      case 4: v += c[0] * exp(c[1] * x[2]) * cos(c[2] * x[0]) * sin(c[3] * x[1]); break;
      case 5: v += c[0] * exp(c[1] * x[dim - 1]) * cos(c[2] * x[0]); break;
      default: break;
    }
    p += 2 + nc;
  }
  return v;
}

static int fn_is_zero(const double* spec) { return spec == NULL || (int)spec[0] == 0; }

/* Gradient of a problem function, term by term by the rules of calculus     */
/* (the Neumann data of a mixed problem is given as h = n . grad phi).      */
static double dpow(double x, int e) { return e == 0 ? 0.0 : e * ipow(x, e - 1); }

void orc_fn_grad(const double* spec, int dim, const double* x, double* grad) {
  for (int a = 0; a < dim; ++a) grad[a] = 0.0;
  const int nt = (int)spec[0];
  const double* p = spec + 1;
  for (int t = 0; t < nt; ++t) {
    const int kind = (int)p[0], nc = (int)p[1];
    const double* c = p + 2;
    if (kind == 1) {
      int idx = 0;
      for (int tt = 0; tt <= 4 && idx < nc; ++tt) {
        if (dim == 2) {
          for (int i = tt; i >= 0 && idx < nc; --i, ++idx) {
            const int j = tt - i;
            grad[0] += c[idx] * dpow(x[0], i) * ipow(x[1], j);
            grad[1] += c[idx] * ipow(x[0], i) * dpow(x[1], j);
          }
        } else {
          for (int i = tt; i >= 0 && idx < nc; --i)
            for (int j = tt - i; j >= 0 && idx < nc; --j, ++idx) {
              const int k = tt - i - j;
              grad[0] += c[idx] * dpow(x[0], i) * ipow(x[1], j) * ipow(x[2], k);
              grad[1] += c[idx] * ipow(x[0], i) * dpow(x[1], j) * ipow(x[2], k);
              grad[2] += c[idx] * ipow(x[0], i) * ipow(x[1], j) * dpow(x[2], k);
            }
        }
      }
    } else if (kind == 2 || kind == 3) {
      /* GAUSS: A e(r2), e = exp(-r2/(2 s^2)), grad = -A e d / s^2 (d = x - c); */
      /* GAUSS_LAPLACIAN: A q e with q = r2/s^4 - dim/s^2,                       */
      /* grad = A e d (2/s^4 - q/s^2)                                            */
      const double sg = c[0];
      const int per = 1 + dim;
      for (int k = 0; 1 + (k + 1) * per <= nc; ++k) {
        const double* b = c + 1 + k * per;
        double d[3] = {0, 0, 0}, r2 = 0.0;
        for (int a = 0; a < dim; ++a) {
          d[a] = x[a] - b[1 + a];
          r2 += d[a] * d[a];
        }
        const double e = exp(-r2 / (2.0 * sg * sg));
        const double s2 = sg * sg, s4 = s2 * s2;
        const double fac = kind == 2 ? -b[0] * e / s2 : b[0] * e * (2.0 / s4 - (r2 / s4 - dim / s2) / s2);
        for (int a = 0; a < dim; ++a) grad[a] += fac * d[a];
      }
    } else if (kind == 4 && dim == 3) {
      const double e = c[0] * exp(c[1] * x[2]);
      grad[0] += -c[2] * e * sin(c[2] * x[0]) * sin(c[3] * x[1]);
      grad[1] += c[3] * e * cos(c[2] * x[0]) * cos(c[3] * x[1]);
      grad[2] += c[1] * e * cos(c[2] * x[0]) * sin(c[3] * x[1]);
    } else if (kind == 5) {
      const double e = c[0] * exp(c[1] * x[dim - 1]);
      grad[0] += -c[2] * e * sin(c[2] * x[0]);
      grad[dim - 1] += c[1] * e * cos(c[2] * x[0]);
    }
    p += 2 + nc;
  }
}

/* Neumann data h(z) = hv(z) + n . grad hp(z) (either part may be empty).  */
double orc_neumann_eval(const double* hv, const double* hp, int dim, const double* z, const double* n) {
  double v = fn_is_zero(hv) ? 0.0 : orc_fn_eval(hv, dim, z);
  if (!fn_is_zero(hp)) {
    double g[3];
    orc_fn_grad(hp, dim, z, g);
    for (int a = 0; a < dim; ++a) v += n[a] * g[a];
  }
  return v;
}

/* ------------------------------------------------------------------------ */
/* Free-space Green's function of the Laplacian and its derivatives, App. A. */
/* d = y - x, r = |d|.  out = [G, dG/dx (dim), dG/dn_y, d2G/dx dn_y (dim)].  */
/* ------------------------------------------------------------------------ */
void orc_green(int dim, const double* x, const double* y, const double* ny, double* out) {
  double d[3] = {0, 0, 0}, r2 = 0.0, nd = 0.0;
  for (int a = 0; a < dim; ++a) {
    d[a] = y[a] - x[a];
    r2 += d[a] * d[a];
    nd += ny[a] * d[a];
  }
  const double r = sqrt(r2);
  if (dim == 2) {
    out[0] = log(r) / (2.0 * ORC_PI);
    for (int a = 0; a < 2; ++a) out[1 + a] = -d[a] / (2.0 * ORC_PI * r2);
    out[3] = nd / (2.0 * ORC_PI * r2);
    for (int a = 0; a < 2; ++a)
      out[4 + a] = 2.0 * nd * d[a] / (2.0 * ORC_PI * r2 * r2) - ny[a] / (2.0 * ORC_PI * r2);
  } else {
    const double r3 = r2 * r, r5 = r3 * r2;
    out[0] = -1.0 / (4.0 * ORC_PI * r);
    for (int a = 0; a < 3; ++a) out[1 + a] = -d[a] / (4.0 * ORC_PI * r3);
    out[4] = nd / (4.0 * ORC_PI * r3);
    for (int a = 0; a < 3; ++a) out[5 + a] = 3.0 * nd * d[a] / (4.0 * ORC_PI * r5) - ny[a] / (4.0 * ORC_PI * r3);
  }
}

/* ------------------------------------------------------------------------ */
/* Modified Bessel functions (screened Poisson, App. A), FP64.               */
/* I_n(t), n = 0, 1: the power series sum_k (t/2)^(2k+n) / (k! (k+n)!)     */
/* (DLMF 10.25.2), all terms positive, for t <= 50; above, the integral     */
/* (1/pi) int_0^pi exp(t cos s) cos(n s) ds (DLMF 10.32.3) by the           */
/* trapezoidal rule, exact to rounding for this periodic analytic integrand. */
/* K_n(t): for t <= 2 the series DLMF 10.31.1/10.31.2 with digamma values   */
/* psi(k+1) = -gamma + H_k; above, int_0^inf exp(-t cosh s) cosh(n s) ds    */
/* (DLMF 10.32.9) by the trapezoidal rule with step 1/16, which converges   */
/* exponentially for this analytic, double-exponentially decaying integrand. */
/* ------------------------------------------------------------------------ */
#define ORC_EULER_GAMMA 0.57721566490153286061
double orc_bessel_i(int n, double t) {
  if (t <= 50.0) {
    const double q = 0.25 * t * t;
    double term = n == 0 ? 1.0 : 0.5 * t, sum = term;
    for (int k = 1; k < 300; ++k) {
      term *= q / ((double)k * (double)(k + n));
      sum += term;
      if (term < 1e-18 * sum) break;
    }
    return sum;
  }
  const int m = 512;
  double sum = 0.0;
  for (int j = 0; j <= m; ++j) {
    const double sj = ORC_PI * j / m;
    const double w = (j == 0 || j == m) ? 0.5 : 1.0;
    sum += w * exp(t * cos(sj)) * cos(n * sj);
  }
  return sum / m;
}

double orc_bessel_k(int n, double t) {
  if (t <= 2.0) {
    const double q = 0.25 * t * t, lg = log(0.5 * t);
    double term = 1.0, h = 0.0, sum = 0.0;
    if (n == 0) {
      for (int k = 0; k < 200; ++k) {
        if (k > 0) {
          term *= q / ((double)k * (double)k);
          h += 1.0 / k;
        }
        sum += term * (h - ORC_EULER_GAMMA);
        if (k > 2 && term < 1e-20) break;
      }
      return -lg * orc_bessel_i(0, t) + sum;
    }
    /* n = 1: 1/t + ln(t/2) I_1(t) - (t/4) sum_k (psi(k+1) + psi(k+2)) q^k / (k! (k+1)!) */
    double h1 = 1.0; /* H_(k+1) */
    for (int k = 0; k < 200; ++k) {
      if (k > 0) {
        term *= q / ((double)k * (double)(k + 1));
        h += 1.0 / k;
        h1 += 1.0 / (k + 1);
      }
      sum += term * ((h - ORC_EULER_GAMMA) + (h1 - ORC_EULER_GAMMA));
      if (k > 2 && term < 1e-20) break;
    }
    return 1.0 / t + lg * orc_bessel_i(1, t) - 0.25 * t * sum;
  }
  const double hstep = 1.0 / 16.0;
  double sum = 0.5 * exp(-t);
  for (int j = 1; j < 100000; ++j) {
    const double sj = j * hstep;
    const double v = exp(-t * cosh(sj)) * cosh(n * sj);
    sum += v;
    if (v < 1e-300 || v < 1e-20 * sum) break;
  }
  return sum * hstep;
}

/* Screened Poisson (Delta - sigma) Green's functions, App. A, with k =     */
/* sqrt(sigma): G = -K0(kr)/(2 pi) (2D), -exp(-kr)/(4 pi r) (3D) -- the    */
/* signs that make the printed gradients (Q times the Laplace gradients)    */
/* their derivatives and (Delta - sigma) G = +delta -- so that Eq. 2 keeps  */
/* its form.  Q = kr K1(kr) (2D), exp(-kr)(kr + 1) (3D); grad_x Q =          */
/* k^2 K0(kr) d (2D), k^2 exp(-kr) d (3D).  out as orc_green.               */
void orc_green_sigma(int dim, double k, const double* x, const double* y, const double* ny, double* out) {
  if (!(k > 0.0)) {
    orc_green(dim, x, y, ny, out);
    return;
  }
  double d[3] = {0, 0, 0}, r2 = 0.0, nd = 0.0;
  for (int a = 0; a < dim; ++a) {
    d[a] = y[a] - x[a];
    r2 += d[a] * d[a];
    nd += ny[a] * d[a];
  }
  const double r = sqrt(r2), t = k * r;
  double G0[8];
  orc_green(dim, x, y, ny, G0);
  double Q, gq, Gs;
  if (dim == 2) {
    const double k0 = orc_bessel_k(0, t);
    Q = t * orc_bessel_k(1, t);
    gq = k * k * k0;
    Gs = -k0 / (2.0 * ORC_PI);
  } else {
    const double e = exp(-t);
    Q = e * (t + 1.0);
    gq = k * k * e;
    Gs = -e / (4.0 * ORC_PI * r);
  }
  out[0] = Gs;
  for (int a = 0; a < dim; ++a) out[1 + a] = Q * G0[1 + a];
  out[1 + dim] = Q * G0[1 + dim];
  for (int a = 0; a < dim; ++a) out[2 + dim + a] = Q * G0[2 + dim + a] + G0[1 + dim] * gq * d[a];
}

/* The walk's screened factors for a ball of radius R (t = R sqrt(sigma)):   */
/* the mean over the sphere of a solution of (Delta - sigma) u = 0 is       */
/* u(centre) / C(t), so u(x) = C(t) avg u with C = t / sinh t (3D),          */
/* 1 / I0(t) (2D); its dipole moment gives grad u(x) = (d/R) Qg(t) avg[u nu]  */
/* with Qg = t^3 / (3 (t cosh t - sinh t)) (3D), t / (2 I1(t)) (2D)           */
/* (from the regular solutions i_l, I_m of the expansion about the centre). */
void orc_screened_factors(int dim, double t, double* C, double* Qg) {
  if (!(t > 0.0)) {
    *C = 1.0;
    *Qg = 1.0;
    return;
  }
  if (dim == 2) {
    *C = 1.0 / orc_bessel_i(0, t);
    *Qg = t / (2.0 * orc_bessel_i(1, t));
  } else {
    *C = t < 1e-4 ? 1.0 / (1.0 + t * t / 6.0) : t / sinh(t);
    if (t < 0.5) {
      const double t2 = t * t;
      *Qg = 1.0 / (1.0 + t2 / 10.0 + t2 * t2 / 280.0 + t2 * t2 * t2 / 15120.0 + t2 * t2 * t2 * t2 / 1330560.0);
    } else {
      *Qg = t * t * t / (3.0 * (t * cosh(t) - sinh(t)));
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Geometry: closest point on a segment / triangle, FP64.                    */
/* Triangle: Voronoi-region method (Ericson, Real-Time Collision Detection,  */
/* Sec. 5.1.5).  Each returns the squared distance and the closest point.    */
/* ------------------------------------------------------------------------ */
static double seg_closest64(const double* a, const double* b, const double* p, double* c) {
  const double abx = b[0] - a[0], aby = b[1] - a[1];
  const double apx = p[0] - a[0], apy = p[1] - a[1];
  const double num = apx * abx + apy * aby, den = abx * abx + aby * aby;
  double t = num <= 0.0 ? 0.0 : (num >= den ? 1.0 : num / den);
  c[0] = a[0] + t * abx;
  c[1] = a[1] + t * aby;
  const double dx = p[0] - c[0], dy = p[1] - c[1];
  return dx * dx + dy * dy;
}

static double dot3d(const double* u, const double* v) { return u[0] * v[0] + u[1] * v[1] + u[2] * v[2]; }

/* The same for a segment in 3D (an edge of a triangle mesh). */
static double seg3_closest64(const double* a, const double* b, const double* p, double* c) {
  double ab[3], ap[3];
  for (int k = 0; k < 3; ++k) {
    ab[k] = b[k] - a[k];
    ap[k] = p[k] - a[k];
  }
  const double num = dot3d(ap, ab), den = dot3d(ab, ab);
  const double t = num <= 0.0 ? 0.0 : (num >= den ? 1.0 : num / den);
  double s = 0.0;
  for (int k = 0; k < 3; ++k) {
    c[k] = a[k] + t * ab[k];
    s += (p[k] - c[k]) * (p[k] - c[k]);
  }
  return s;
}

static double tri_closest64(const double* a, const double* b, const double* cc, const double* p, double* c) {
  double ab[3], ac[3], ap[3], bp[3], cp[3];
  for (int i = 0; i < 3; ++i) {
    ab[i] = b[i] - a[i];
    ac[i] = cc[i] - a[i];
    ap[i] = p[i] - a[i];
  }
  const double d1 = dot3d(ab, ap), d2 = dot3d(ac, ap);
  if (d1 <= 0.0 && d2 <= 0.0) {
    memcpy(c, a, 3 * sizeof(double));
    goto done;
  }
  for (int i = 0; i < 3; ++i) bp[i] = p[i] - b[i];
  const double d3 = dot3d(ab, bp), d4 = dot3d(ac, bp);
  if (d3 >= 0.0 && d4 <= d3) {
    memcpy(c, b, 3 * sizeof(double));
    goto done;
  }
  const double vc = d1 * d4 - d3 * d2;
  if (vc <= 0.0 && d1 >= 0.0 && d3 <= 0.0) {
    const double v = d1 / (d1 - d3);
    for (int i = 0; i < 3; ++i) c[i] = a[i] + v * ab[i];
    goto done;
  }
  for (int i = 0; i < 3; ++i) cp[i] = p[i] - cc[i];
  const double d5 = dot3d(ab, cp), d6 = dot3d(ac, cp);
  if (d6 >= 0.0 && d5 <= d6) {
    memcpy(c, cc, 3 * sizeof(double));
    goto done;
  }
  const double vb = d5 * d2 - d1 * d6;
  if (vb <= 0.0 && d2 >= 0.0 && d6 <= 0.0) {
    const double w = d2 / (d2 - d6);
    for (int i = 0; i < 3; ++i) c[i] = a[i] + w * ac[i];
    goto done;
  }
  const double va = d3 * d6 - d5 * d4;
  if (va <= 0.0 && (d4 - d3) >= 0.0 && (d5 - d6) >= 0.0) {
    const double w = (d4 - d3) / ((d4 - d3) + (d5 - d6));
    for (int i = 0; i < 3; ++i) c[i] = b[i] + w * (cc[i] - b[i]);
    goto done;
  }
  {
    const double denom = 1.0 / (va + vb + vc);
    const double v = vb * denom, w = vc * denom;
    for (int i = 0; i < 3; ++i) c[i] = a[i] + ab[i] * v + ac[i] * w;
  }
done : {
  double s = 0.0;
  for (int i = 0; i < 3; ++i) s += (p[i] - c[i]) * (p[i] - c[i]);
  return s;
}
}

typedef struct {
  int dim;
  int64_t nv, np;
  double* V;   /* nv x dim */
  int32_t* F;  /* np x dim vertex indices */
} mesh_t;

static double prim_closest64(const mesh_t* m, int64_t e, const double* p, double* c) {
  const int32_t* f = m->F + e * m->dim;
  if (m->dim == 2) return seg_closest64(m->V + 2 * f[0], m->V + 2 * f[1], p, c);
  return tri_closest64(m->V + 3 * f[0], m->V + 3 * f[1], m->V + 3 * f[2], p, c);
}

/* Brute force over every primitive; ties go to the lowest index. */
void orc_closest_brute64(int dim, const float* V, int64_t nv, const int32_t* F, int64_t np, const double* pts,
                         int64_t n, double* dist, int32_t* prim, double* cp) {
  mesh_t m = {dim, nv, np, NULL, (int32_t*)F};
  m.V = (double*)malloc(sizeof(double) * nv * dim);
  for (int64_t i = 0; i < nv * dim; ++i) m.V[i] = V[i];
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t q = 0; q < n; ++q) {
    double best = INFINITY, c[3], bc[3] = {0, 0, 0};
    int32_t bi = -1;
    for (int64_t e = 0; e < np; ++e) {
      const double d2 = prim_closest64(&m, e, pts + q * dim, c);
      if (d2 < best) {
        best = d2;
        bi = (int32_t)e;
        memcpy(bc, c, sizeof(c));
      }
    }
    dist[q] = sqrt(best);
    prim[q] = bi;
    if (cp) memcpy(cp + q * dim, bc, sizeof(double) * dim);
  }
  free(m.V);
}

/* ------------------------------------------------------------------------ */
/* Canonical FP32 closest-point distances.  Fixed operation order with      */
/* explicit fmaf; the primitive is (a, ab = b-a, [ac = c-a]) in FP32.        */
/* Segment: with num = ab.ap, den = |ab|^2 and inv = 1/den (one FP32         */
/* division per segment): |ap|^2 if num <= 0, |ap-ab|^2 if num >= den, else  */
/* cross(ap,ab)^2 * inv.  Triangle: Ericson's Voronoi regions.  Used only to */
/* check the GPU's primitive index bit-exactly.                             */
/* ------------------------------------------------------------------------ */
static float seg_d2_f32(float ax, float ay, float abx, float aby, float inv, float px, float py) {
  const float apx = px - ax, apy = py - ay;
  const float num = fmaf(apy, aby, apx * abx);
  const float den = fmaf(aby, aby, abx * abx);
  if (num <= 0.0f) return fmaf(apy, apy, apx * apx);
  if (num >= den) {
    const float bx = apx - abx, by = apy - aby;
    return fmaf(by, by, bx * bx);
  }
  const float c = fmaf(apx, aby, -(apy * abx));
  return (c * c) * inv;
}

static float dot3f(const float* u, const float* v) { return fmaf(u[2], v[2], fmaf(u[1], v[1], u[0] * v[0])); }

static float tri_d2_f32(const float* a, const float* ab, const float* ac, const float* p) {
  float ap[3], bp[3], cp[3], df[3];
  for (int i = 0; i < 3; ++i) ap[i] = p[i] - a[i];
  const float d1 = dot3f(ab, ap), d2 = dot3f(ac, ap);
  if (d1 <= 0.0f && d2 <= 0.0f) return dot3f(ap, ap);
  for (int i = 0; i < 3; ++i) bp[i] = ap[i] - ab[i];
  const float d3 = dot3f(ab, bp), d4 = dot3f(ac, bp);
  if (d3 >= 0.0f && d4 <= d3) return dot3f(bp, bp);
  const float vc = fmaf(d1, d4, -(d3 * d2));
  if (vc <= 0.0f && d1 >= 0.0f && d3 <= 0.0f) {
    const float v = d1 / (d1 - d3);
    for (int i = 0; i < 3; ++i) df[i] = fmaf(-v, ab[i], ap[i]);
    return dot3f(df, df);
  }
  for (int i = 0; i < 3; ++i) cp[i] = ap[i] - ac[i];
  const float d5 = dot3f(ab, cp), d6 = dot3f(ac, cp);
  if (d6 >= 0.0f && d5 <= d6) return dot3f(cp, cp);
  const float vb = fmaf(d5, d2, -(d1 * d6));
  if (vb <= 0.0f && d2 >= 0.0f && d6 <= 0.0f) {
    const float w = d2 / (d2 - d6);
    for (int i = 0; i < 3; ++i) df[i] = fmaf(-w, ac[i], ap[i]);
    return dot3f(df, df);
  }
  const float va = fmaf(d3, d6, -(d5 * d4));
  const float e43 = d4 - d3, e56 = d5 - d6;
  if (va <= 0.0f && e43 >= 0.0f && e56 >= 0.0f) {
    const float w = e43 / (e43 + e56);
    for (int i = 0; i < 3; ++i) df[i] = fmaf(-w, ac[i] - ab[i], bp[i]);
    return dot3f(df, df);
  }
  const float denom = 1.0f / (va + vb + vc);
  const float v = vb * denom, w = vc * denom;
  for (int i = 0; i < 3; ++i) df[i] = fmaf(-w, ac[i], fmaf(-v, ab[i], ap[i]));
  return dot3f(df, df);
}

/* FP32 brute-force argmin of the canonical squared distance; ties -> lowest index. */
void orc_closest_brute32(int dim, const float* V, int64_t nv, const int32_t* F, int64_t np, const float* pts,
                         int64_t n, float* d2_out, int32_t* prim) {
  (void)nv;
  float* P = (float*)malloc(sizeof(float) * np * 9);
  for (int64_t e = 0; e < np; ++e) {
    const int32_t* f = F + e * dim;
    for (int a = 0; a < dim; ++a) {
      const float va = V[(int64_t)f[0] * dim + a];
      P[e * 9 + a] = va;
      P[e * 9 + 3 + a] = V[(int64_t)f[1] * dim + a] - va;
      if (dim == 3) P[e * 9 + 6 + a] = V[(int64_t)f[2] * dim + a] - va;
    }
    if (dim == 2) P[e * 9 + 6] = 1.0f / fmaf(P[e * 9 + 4], P[e * 9 + 4], P[e * 9 + 3] * P[e * 9 + 3]);
  }
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t q = 0; q < n; ++q) {
    float best = INFINITY;
    int32_t bi = -1;
    const float* p = pts + q * dim;
    for (int64_t e = 0; e < np; ++e) {
      const float* r = P + e * 9;
      const float d2 = dim == 2 ? seg_d2_f32(r[0], r[1], r[3], r[4], r[6], p[0], p[1]) : tri_d2_f32(r, r + 3, r + 6, p);
      if (d2 < best) {
        best = d2;
        bi = (int32_t)e;
      }
    }
    d2_out[q] = best;
    prim[q] = bi;
  }
  free(P);
}

/* Canonical FP32 crossing-number inside test (2D polygon, +x ray). */
static int inside2d_f32(const float* V, const int32_t* F, int64_t np, float px, float py) {
  int c = 0;
  for (int64_t e = 0; e < np; ++e) {
    const float ax = V[2 * F[2 * e]], ay = V[2 * F[2 * e] + 1];
    const float bx = V[2 * F[2 * e + 1]], by = V[2 * F[2 * e + 1] + 1];
    if ((ay > py) != (by > py)) {
      const float t = (py - ay) / (by - ay);
      const float xi = fmaf(t, bx - ax, ax);
      if (px < xi) c ^= 1;
    }
  }
  return c;
}

void orc_inside2d_f32(const float* V, const int32_t* F, int64_t np, const float* pts, int64_t n, int32_t* out) {
#pragma omp parallel for schedule(static)
  for (int64_t q = 0; q < n; ++q) out[q] = inside2d_f32(V, F, np, pts[2 * q], pts[2 * q + 1]);
}

/* ------------------------------------------------------------------------ */
/* A plain FP64 BVH (median split on the longest centroid axis) so that the */
/* oracle's walks finish on large meshes.  The query returns exactly what   */
/* the brute force above returns (checked in the tests).                    */
/* ------------------------------------------------------------------------ */
typedef struct {
  double lo[3], hi[3];
  int64_t left, right; /* children, or -1 */
  int64_t start, count;
} bnode_t;

typedef struct {
  mesh_t m;
  bnode_t* nodes;
  int64_t n_nodes;
  int64_t* order;
  double* cen;
  double slack;
} obvh_t;

static int g_sort_axis;
static const double* g_sort_cen;
static int cmp_cen(const void* x, const void* y) {
  const double a = g_sort_cen[*(const int64_t*)x * 3 + g_sort_axis];
  const double b = g_sort_cen[*(const int64_t*)y * 3 + g_sort_axis];
  if (a < b) return -1;
  if (a > b) return 1;
  const int64_t ia = *(const int64_t*)x, ib = *(const int64_t*)y;
  return (ia > ib) - (ia < ib);
}

static void prim_box(const mesh_t* m, int64_t e, double* lo, double* hi) {
  const int32_t* f = m->F + e * m->dim;
  for (int a = 0; a < 3; ++a) {
    lo[a] = INFINITY;
    hi[a] = -INFINITY;
  }
  for (int v = 0; v < m->dim; ++v)
    for (int a = 0; a < m->dim; ++a) {
      const double x = m->V[(int64_t)f[v] * m->dim + a];
      if (x < lo[a]) lo[a] = x;
      if (x > hi[a]) hi[a] = x;
    }
  for (int a = m->dim; a < 3; ++a) lo[a] = hi[a] = 0.0;
}

static int64_t bvh_build_rec(obvh_t* b, int64_t start, int64_t count) {
  const int64_t id = b->n_nodes++;
  bnode_t* nd = &b->nodes[id];
  for (int a = 0; a < 3; ++a) {
    nd->lo[a] = INFINITY;
    nd->hi[a] = -INFINITY;
  }
  double clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t i = start; i < start + count; ++i) {
    double lo[3], hi[3];
    prim_box(&b->m, b->order[i], lo, hi);
    for (int a = 0; a < 3; ++a) {
      if (lo[a] < nd->lo[a]) nd->lo[a] = lo[a];
      if (hi[a] > nd->hi[a]) nd->hi[a] = hi[a];
      const double c = b->cen[b->order[i] * 3 + a];
      if (c < clo[a]) clo[a] = c;
      if (c > chi[a]) chi[a] = c;
    }
  }
  nd->start = start;
  nd->count = count;
  nd->left = nd->right = -1;
  if (count <= 4) return id;
  int axis = 0;
  for (int a = 1; a < b->m.dim; ++a)
    if (chi[a] - clo[a] > chi[axis] - clo[axis]) axis = a;
  g_sort_axis = axis;
  g_sort_cen = b->cen;
  qsort(b->order + start, (size_t)count, sizeof(int64_t), cmp_cen);
  const int64_t half = count / 2;
  const int64_t l = bvh_build_rec(b, start, half);
  const int64_t r = bvh_build_rec(b, start + half, count - half);
  b->nodes[id].left = l;
  b->nodes[id].right = r;
  return id;
}

void* orc_bvh_create(int dim, const float* V, int64_t nv, const int32_t* F, int64_t np) {
  obvh_t* b = (obvh_t*)calloc(1, sizeof(obvh_t));
  b->m.dim = dim;
  b->m.nv = nv;
  b->m.np = np;
  b->m.V = (double*)malloc(sizeof(double) * nv * dim);
  for (int64_t i = 0; i < nv * dim; ++i) b->m.V[i] = V[i];
  b->m.F = (int32_t*)malloc(sizeof(int32_t) * np * dim);
  memcpy(b->m.F, F, sizeof(int32_t) * np * dim);
  b->order = (int64_t*)malloc(sizeof(int64_t) * np);
  b->cen = (double*)calloc((size_t)np * 3, sizeof(double));
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t e = 0; e < np; ++e) {
    b->order[e] = e;
    const int32_t* f = b->m.F + e * dim;
    for (int a = 0; a < dim; ++a) {
      double s = 0.0;
      for (int v = 0; v < dim; ++v) s += b->m.V[(int64_t)f[v] * dim + a];
      b->cen[e * 3 + a] = s / dim;
    }
  }
  for (int64_t i = 0; i < nv * dim; ++i) {
    const int a = (int)(i % dim);
    if (b->m.V[i] < lo[a]) lo[a] = b->m.V[i];
    if (b->m.V[i] > hi[a]) hi[a] = b->m.V[i];
  }
  double diag = 0.0;
  for (int a = 0; a < dim; ++a) diag += (hi[a] - lo[a]) * (hi[a] - lo[a]);
  b->slack = 1e-12 * sqrt(diag);
  b->nodes = (bnode_t*)malloc(sizeof(bnode_t) * (2 * np + 1));
  b->n_nodes = 0;
  if (np > 0) bvh_build_rec(b, 0, np);
  return b;
}

void orc_bvh_free(void* h) {
  obvh_t* b = (obvh_t*)h;
  if (!b) return;
  free(b->m.V);
  free(b->m.F);
  free(b->order);
  free(b->cen);
  free(b->nodes);
  free(b);
}

static double box_d2(const bnode_t* n, const double* p, int dim) {
  double s = 0.0;
  for (int a = 0; a < dim; ++a) {
    double d = 0.0;
    if (p[a] < n->lo[a])
      d = n->lo[a] - p[a];
    else if (p[a] > n->hi[a])
      d = p[a] - n->hi[a];
    s += d * d;
  }
  return s;
}

/* Closest primitive: nodes are skipped only when their box is farther than */
/* the best distance plus a tiny slack, so ties and rounding never prune    */
/* the true minimum; ties go to the lowest primitive index.                 */
static double bvh_closest(const obvh_t* b, const double* p, double* cbest, int64_t* ibest) {
  double best = INFINITY, bd = INFINITY;
  int64_t bi = -1;
  int64_t stack[128];
  int sp = 0;
  if (b->n_nodes) stack[sp++] = 0;
  const int dim = b->m.dim;
  while (sp) {
    const bnode_t* n = &b->nodes[stack[--sp]];
    const double lim = bd + b->slack;
    if (box_d2(n, p, dim) > lim * lim) continue;
    if (n->left < 0) {
      for (int64_t i = n->start; i < n->start + n->count; ++i) {
        const int64_t e = b->order[i];
        double c[3];
        const double d2 = prim_closest64(&b->m, e, p, c);
        if (d2 < best || (d2 == best && e < bi)) {
          best = d2;
          bd = sqrt(d2);
          bi = e;
          memcpy(cbest, c, sizeof(double) * dim);
        }
      }
    } else {
      const double dl = box_d2(&b->nodes[n->left], p, dim), dr = box_d2(&b->nodes[n->right], p, dim);
      if (dl <= dr) {
        stack[sp++] = n->right;
        stack[sp++] = n->left;
      } else {
        stack[sp++] = n->left;
        stack[sp++] = n->right;
      }
    }
  }
  *ibest = bi;
  return best;
}

void orc_bvh_closest(void* h, const double* pts, int64_t n, double* dist, int32_t* prim, double* cp) {
  const obvh_t* b = (const obvh_t*)h;
  const int dim = b->m.dim;
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t q = 0; q < n; ++q) {
    double c[3];
    int64_t e;
    const double d2 = bvh_closest(b, pts + q * dim, c, &e);
    dist[q] = sqrt(d2);
    prim[q] = (int32_t)e;
    if (cp) memcpy(cp + q * dim, c, sizeof(double) * dim);
  }
}

/* ------------------------------------------------------------------------ */
/* Element measures, outward normals and the boundary sampler (Sec. 4       */
/* "Sampling"; Alg. 1 draws z, n_z ~ p on the boundary; Sec. 3.2 moves the  */
/* Dirichlet samples inward by l along the element normal).                 */
/* Polygons are counter-clockwise, triangles wind counter-clockwise seen    */
/* from outside, so the outward normal of a->b is (dy, -dx)/len in 2D and   */
/* (b-a)x(c-a)/|.| in 3D.                                                    */
/* ------------------------------------------------------------------------ */
static double elem_measure_normal(int dim, const float* V, const int32_t* f, double* nrm) {
  if (dim == 2) {
    const double ax = V[2 * f[0]], ay = V[2 * f[0] + 1], bx = V[2 * f[1]], by = V[2 * f[1] + 1];
    const double dx = bx - ax, dy = by - ay;
    const double len = sqrt(dx * dx + dy * dy);
    nrm[0] = dy / len;
    nrm[1] = -dx / len;
    return len;
  }
  double e1[3], e2[3], c[3];
  for (int a = 0; a < 3; ++a) {
    e1[a] = (double)V[3 * f[1] + a] - (double)V[3 * f[0] + a];
    e2[a] = (double)V[3 * f[2] + a] - (double)V[3 * f[0] + a];
  }
  c[0] = e1[1] * e2[2] - e1[2] * e2[1];
  c[1] = e1[2] * e2[0] - e1[0] * e2[2];
  c[2] = e1[0] * e2[1] - e1[1] * e2[0];
  const double len = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
  for (int a = 0; a < 3; ++a) nrm[a] = c[a] / len;
  return 0.5 * len;
}

/* Total boundary measure |dOmega| as the sequential sum of element measures. */
double orc_boundary_measure(int dim, const float* V, const int32_t* F, int64_t np) {
  double s = 0.0, n[3];
  for (int64_t e = 0; e < np; ++e) s += elem_measure_normal(dim, V, F + e * dim, n);
  return s;
}

/* Measure and outward unit normal of an element given by FP64 vertex       */
/* positions P[0..dim-1], in the same operation order as                    */
/* elem_measure_normal (so P = the mesh's own vertices gives the same bits).*/
static double pts_measure_normal(int dim, double P[3][3], double* nrm) {
  if (dim == 2) {
    const double dx = P[1][0] - P[0][0], dy = P[1][1] - P[0][1];
    const double len = sqrt(dx * dx + dy * dy);
    nrm[0] = dy / len;
    nrm[1] = -dx / len;
    return len;
  }
  double e1[3], e2[3], c[3];
  for (int a = 0; a < 3; ++a) {
    e1[a] = P[1][a] - P[0][a];
    e2[a] = P[2][a] - P[0][a];
  }
  c[0] = e1[1] * e2[2] - e1[2] * e2[1];
  c[1] = e1[2] * e2[0] - e1[0] * e2[2];
  c[2] = e1[0] * e2[1] - e1[1] * e2[0];
  const double len = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
  for (int a = 0; a < 3; ++a) nrm[a] = c[a] / len;
  return 0.5 * len;
}

/* ------------------------------------------------------------------------ */
/* The offset Dirichlet boundary (Sec. 3.2, Fig. "Dirichlet offset          */
/* boundary"): the cache's samples lie on the boundary of a CLOSED region   */
/* inside Omega, about l from the boundary, and the BIE (Eq. 2) and the     */
/* source samples refer to that region.  Reading: the region is bounded by  */
/* the mesh with every vertex v moved to v - l m_v, m_v built from the unit */
/* normals of the MOVED elements at v (all elements, or the Dirichlet ones  */
/* of a mixed boundary, whose Neumann elements stay put):                   */
/*   2D, k = 2 moved segments with normals na, nb, S = na + nb:             */
/*       m = S / max(|S|^2 / 2, 1/4)                                        */
/*     (|S|^2/2 = 1 + na.nb: the miter, both moved segments parallel to     */
/*      theirs at distance exactly l, for turning angles up to 138.6 deg);  */
/*   2D, any other k >= 1: m = S / |S|;                                     */
/*   3D: N = sum over the moved triangles at v of theta_f n_f (theta_f the */
/*       triangle's angle at v, n_f its unit normal: the angle-weighted     */
/*       pseudonormal, independent of how flat parts are triangulated), N^  */
/*       its direction, m = N^ / max(min_f n_f . N^, 1/4), so every moved   */
/*       triangle's plane moves inward by at least l at v (a box corner     */
/*       moves by (1,1,1) l: l from each of its three faces).               */
/* A vertex with no moved element, or S = 0 / N = 0, keeps m = 0.           */
/* fixed (may be NULL): fixed[e] != 0 marks an element that is not moved.   */
/* Returns max_v |m_v| (the reach: the moved mesh lies within l x reach of  */
/* the boundary).                                                            */
/* ------------------------------------------------------------------------ */
double orc_offset_disp(int dim, const float* V, int64_t nv, const int32_t* F, int64_t np, const uint8_t* fixed,
                       double* m) {
  int32_t* cnt = (int32_t*)calloc((size_t)nv, sizeof(int32_t));
  double* S = (double*)calloc((size_t)nv * dim, sizeof(double));
  for (int64_t i = 0; i < nv * dim; ++i) m[i] = 0.0;
  for (int64_t e = 0; e < np; ++e) {
    if (fixed && fixed[e]) continue;
    const int32_t* f = F + e * dim;
    double n[3];
    if (dim == 2) {
      elem_measure_normal(2, V, f, n);
      for (int k = 0; k < 2; ++k) {
        S[2 * (int64_t)f[k]] += n[0];
        S[2 * (int64_t)f[k] + 1] += n[1];
        cnt[f[k]] += 1;
      }
    } else {
      elem_measure_normal(3, V, f, n);
      for (int k = 0; k < 3; ++k) {
        /* angle at corner k between the edges to the other two corners */
        double p[3], q[3];
        for (int a = 0; a < 3; ++a) {
          p[a] = (double)V[3 * f[(k + 1) % 3] + a] - (double)V[3 * f[k] + a];
          q[a] = (double)V[3 * f[(k + 2) % 3] + a] - (double)V[3 * f[k] + a];
        }
        const double x[3] = {p[1] * q[2] - p[2] * q[1], p[2] * q[0] - p[0] * q[2], p[0] * q[1] - p[1] * q[0]};
        const double th = atan2(sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]), p[0] * q[0] + p[1] * q[1] + p[2] * q[2]);
        for (int a = 0; a < 3; ++a) S[3 * (int64_t)f[k] + a] += th * n[a];
        cnt[f[k]] += 1;
      }
    }
  }
  if (dim == 2) {
    for (int64_t v = 0; v < nv; ++v) {
      const double s0 = S[2 * v], s1 = S[2 * v + 1];
      const double q = s0 * s0 + s1 * s1;
      if (cnt[v] == 0 || !(q > 0.0)) continue;
      const double den = cnt[v] == 2 ? fmax(0.5 * q, 0.25) : sqrt(q);
      m[2 * v] = s0 / den;
      m[2 * v + 1] = s1 / den;
    }
  } else {
    double* cmin = (double*)malloc(sizeof(double) * (size_t)nv);
    for (int64_t v = 0; v < nv; ++v) {
      cmin[v] = 2.0;
      const double q = sqrt(S[3 * v] * S[3 * v] + S[3 * v + 1] * S[3 * v + 1] + S[3 * v + 2] * S[3 * v + 2]);
      if (q > 0.0)
        for (int a = 0; a < 3; ++a) S[3 * v + a] = S[3 * v + a] / q;
      else
        cnt[v] = 0;
    }
    for (int64_t e = 0; e < np; ++e) {
      if (fixed && fixed[e]) continue;
      const int32_t* f = F + e * 3;
      double n[3];
      elem_measure_normal(3, V, f, n);
      for (int k = 0; k < 3; ++k) {
        const double* Nv = S + 3 * (int64_t)f[k];
        const double c = n[0] * Nv[0] + n[1] * Nv[1] + n[2] * Nv[2];
        if (c < cmin[f[k]]) cmin[f[k]] = c;
      }
    }
    for (int64_t v = 0; v < nv; ++v) {
      if (cnt[v] == 0) continue;
      const double den = fmax(cmin[v], 0.25);
      for (int a = 0; a < 3; ++a) m[3 * v + a] = S[3 * v + a] / den;
    }
    free(cmin);
  }
  double reach = 0.0;
  for (int64_t v = 0; v < nv; ++v) {
    double q = 0.0;
    for (int a = 0; a < dim; ++a) q += m[dim * v + a] * m[dim * v + a];
    if (sqrt(q) > reach) reach = sqrt(q);
  }
  free(cnt);
  free(S);
  return reach;
}

/* The moved mesh's vertices rounded to FP32: V'[v] = fl32(V[v] - l m_v).   */
void orc_offset_vertices(int dim, const float* V, int64_t nv, const double* m, double l, float* Vout) {
  for (int64_t i = 0; i < nv * dim; ++i) Vout[i] = (float)((double)V[i] - l * m[i]);
}

/* N stratified boundary samples.  Sample i draws (u0,u1,u2) from Philox    */
/* (id = i, word2 = 0, tag = 1); s = (i + u0)/N picks the element through   */
/* the CDF of element measures; 2D reuses the position of s inside the      */
/* element's CDF interval as the arclength parameter lam, 3D draws          */
/* barycentrics (1-sqrt(u1), sqrt(u1)(1-u2), sqrt(u1)u2).  The sample sits  */
/* at those coordinates on the MOVED element (vertices P_k = v_k - l m_k,   */
/* see orc_offset_disp): an affine map of the element, so the point stays   */
/* uniform on it.  Its density on the offset surface is                     */
/* 1 / (|dOmega| jac) with jac = |moved element| / |element|, so 1/p =      */
/* |dOmega| jac; nrm is the moved element's outward unit normal.            */
/* With fixed non-NULL, elements e with fixed[e] != 0 (the Neumann part of  */
/* a mixed boundary) are not moved (jac = 1).                               */
static void sample_boundary(int dim, const float* V, const int32_t* F, int64_t np, int64_t N, double l,
                            uint64_t seed, const uint8_t* fixed, const double* m, double* z, double* nrm,
                            double* jac, int32_t* elem) {
  double* cdf = (double*)malloc(sizeof(double) * (np + 1));
  double n[3];
  cdf[0] = 0.0;
  for (int64_t e = 0; e < np; ++e) cdf[e + 1] = cdf[e] + elem_measure_normal(dim, V, F + e * dim, n);
  const double total = cdf[np];
  for (int64_t i = 0; i < N; ++i) {
    double u[4];
    draw(seed, (uint64_t)i, 0u, 1u, u);
    const double s = ((double)i + u[0]) / (double)N;
    const double t = s * total;
    /* smallest e with cdf[e+1] > t */
    int64_t lo = 0, hi = np - 1;
    while (lo < hi) {
      const int64_t mid = (lo + hi) / 2;
      if (cdf[mid + 1] > t)
        hi = mid;
      else
        lo = mid + 1;
    }
    const int64_t e = lo;
    const int32_t* f = F + e * dim;
    const double meas = elem_measure_normal(dim, V, f, n);
    const double le = (fixed && fixed[e]) ? 0.0 : l;
    double P[3][3];
    for (int k = 0; k < dim; ++k)
      for (int a = 0; a < dim; ++a) P[k][a] = (double)V[dim * f[k] + a] - le * m[dim * f[k] + a];
    double nm[3];
    const double meas_m = pts_measure_normal(dim, P, nm);
    double p[3];
    if (dim == 2) {
      double lam = (t - cdf[e]) / meas;
      if (lam < 0.0) lam = 0.0;
      if (lam > 1.0) lam = 1.0;
      for (int a = 0; a < 2; ++a) p[a] = P[0][a] + lam * (P[1][a] - P[0][a]);
    } else {
      const double sq = sqrt(u[1]);
      const double b1 = sq * (1.0 - u[2]), b2 = sq * u[2];
      for (int a = 0; a < 3; ++a) p[a] = P[0][a] + b1 * (P[1][a] - P[0][a]) + b2 * (P[2][a] - P[0][a]);
    }
    for (int a = 0; a < dim; ++a) {
      z[i * dim + a] = p[a];
      nrm[i * dim + a] = nm[a];
    }
    jac[i] = meas_m / meas;
    elem[i] = (int32_t)e;
  }
  free(cdf);
}

void orc_sample_boundary(int dim, const float* V, int64_t nv, const int32_t* F, int64_t np, int64_t N, double l,
                         uint64_t seed, double* z, double* nrm, double* jac, int32_t* elem) {
  double* m = (double*)malloc(sizeof(double) * (size_t)nv * dim);
  orc_offset_disp(dim, V, nv, F, np, NULL, m);
  sample_boundary(dim, V, F, np, N, l, seed, NULL, m, z, nrm, jac, elem);
  free(m);
}

void orc_sample_boundary_mixed(int dim, const float* V, int64_t nv, const int32_t* F, int64_t np, int64_t N,
                               double l, uint64_t seed, const uint8_t* neumann, double* z, double* nrm, double* jac,
                               int32_t* elem) {
  double* m = (double*)malloc(sizeof(double) * (size_t)nv * dim);
  orc_offset_disp(dim, V, nv, F, np, neumann, m);
  sample_boundary(dim, V, F, np, N, l, seed, neumann, m, z, nrm, jac, elem);
  free(m);
}

/* ------------------------------------------------------------------------ */
/* Walk on spheres (Sec. 3.1) for Laplace(u) = f, u = g on the boundary.    */
/*                                                                          */
/* Ball B(x,R), R = distance to the boundary.  With G^B the Green's         */
/* function of -Laplacian on the ball (zero on its sphere):                 */
/*   u(x)      = mean_{sphere} u  -  int_B G^B(x,y) f(y) dy                  */
/*   grad u(x) = (d/R) mean_{sphere}[u(z) nu]  -  int_B grad_x G^B f dy     */
/* (the second is Eq. 7 with the ball's Poisson-kernel derivative at the    */
/* centre).  Step k draws Philox (id = walk id, word2 = k, tag):            */
/*   direction from (u0,u1): 2D (cos 2pi u0, sin 2pi u0); 3D z = 1-2u0,     */
/*   phi = 2pi u1; source point y = x + rho w with rho = R u2 (uniform      */
/*   radius, density 1/(R |S| rho^(d-1))) giving the weights                */
/*     w_u    = -R rho ln(R/rho)    (2D)   or  -rho (R - rho)      (3D)     */
/*     w_grad = -R (1 - (rho/R)^d) w                                         */
/* A walk stops at the first closest-point query with distance < eps       */
/* (eps shell) and returns g at the closest boundary point; it is capped    */
/* after max_steps queries.                                                 */
/* Per walk:  U = g(pbar_end) + sum_k w_u,k f(y_k)                           */
/*            grad = nu0 [ (d/R0)(U - w_u,0 f(y_0) - g(pbar_0)) + w_g,0 ]    */
/* where g(pbar_0), a constant independent of the step-0 direction, is a    */
/* control variate (mean of nu over the sphere is zero).  A walk whose      */
/* start is already inside the shell has grad = 0.                          */
/* ------------------------------------------------------------------------ */
typedef struct {
  const obvh_t* bvh;
  const double* g;
  const double* f;
  double eps;
  int max_steps;
  uint64_t seed;
  uint32_t tag;
  const double* gv; /* vertex values of g, or NULL for the closed form g */
  double sqs;       /* sqrt(sigma) of the screened equation, 0 for Poisson */
} walk_ctx_t;

/* Boundary data given by values at the mesh vertices: g at a point p of   */
/* element e is the linear interpolation of its vertex values -- on a       */
/* segment by the projection parameter t = (p-a).(b-a)/|b-a|^2 clamped to   */
/* [0,1], on a triangle by the barycentric coordinates of p (p on the       */
/* triangle's plane; Ericson, Real-Time Collision Detection, Sec. 3.4).     */
double orc_vertex_interp(const void* bvh, const double* gv, int64_t e, const double* p) {
  const mesh_t* m = &((const obvh_t*)bvh)->m;
  const int32_t* f = m->F + e * m->dim;
  if (m->dim == 2) {
    const double* a = m->V + 2 * (int64_t)f[0];
    const double* b = m->V + 2 * (int64_t)f[1];
    const double abx = b[0] - a[0], aby = b[1] - a[1];
    double t = ((p[0] - a[0]) * abx + (p[1] - a[1]) * aby) / (abx * abx + aby * aby);
    t = fmin(fmax(t, 0.0), 1.0);
    return (1.0 - t) * gv[f[0]] + t * gv[f[1]];
  }
  const double* a = m->V + 3 * (int64_t)f[0];
  const double* b = m->V + 3 * (int64_t)f[1];
  const double* c = m->V + 3 * (int64_t)f[2];
  double v0[3], v1[3], v2[3];
  for (int i = 0; i < 3; ++i) {
    v0[i] = b[i] - a[i];
    v1[i] = c[i] - a[i];
    v2[i] = p[i] - a[i];
  }
  const double d00 = dot3d(v0, v0), d01 = dot3d(v0, v1), d11 = dot3d(v1, v1);
  const double d20 = dot3d(v2, v0), d21 = dot3d(v2, v1);
  const double den = d00 * d11 - d01 * d01;
  const double bv = (d11 * d20 - d01 * d21) / den;
  const double bw = (d00 * d21 - d01 * d20) / den;
  return (1.0 - bv - bw) * gv[f[0]] + bv * gv[f[1]] + bw * gv[f[2]];
}

static double g_at(const walk_ctx_t* w, const double* p, int64_t e) {
  return w->gv ? orc_vertex_interp(w->bvh, w->gv, e, p) : orc_fn_eval(w->g, w->bvh->m.dim, p);
}

/* One sphere step: direction w from (u0,u1) and, for radius R, the source  */
/* point radius rho = R u2 with its weights w_u and the scalar w_g such     */
/* that the step-0 gradient source term is w_g * w.                          */
void orc_sphere_step(int dim, double R, double u0, double u1, double u2, double* om, double* rho, double* wu,
                     double* wg) {
  if (dim == 2) {
    om[0] = cos(2.0 * ORC_PI * u0);
    om[1] = sin(2.0 * ORC_PI * u0);
  } else {
    const double zc = 1.0 - 2.0 * u0, phi = 2.0 * ORC_PI * u1;
    const double s = sqrt(fmax(0.0, 1.0 - zc * zc));
    om[0] = s * cos(phi);
    om[1] = s * sin(phi);
    om[2] = zc;
  }
  const double r = R * u2;
  *rho = r;
  *wu = dim == 2 ? -R * r * log(R / r) : -r * (R - r);
  *wg = -R * (1.0 - ipow(r / R, dim));
}

/* Screened source weights of one step (Delta u - sigma u = f, k = sqrt(   */
/* sigma)).  The ball B(x, R) gives u(x) = C avg_sphere u - int_B G f with  */
/* G the Green's function of (sigma - Delta) on the ball, zero on its       */
/* sphere, seen from the centre (r = |y - x|):                              */
/*   2D  G = [K0(kr) - K0(kR) I0(kr) / I0(kR)] / (2 pi)                     */
/*   3D  G = sinh(k (R - r)) / (4 pi r sinh(kR))                            */
/* (the fundamental solution minus the regular solution that matches it on */
/* the sphere).  Its gradient in the evaluation point at the centre, for    */
/* the gradient estimate, is w phi(r), w = (y - x)/r, with phi the l = 1    */
/* radial mode that has the singular part -d/dr of the fundamental solution */
/* and vanishes at R:                                                       */
/*   2D  phi = k [K1(kr) - K1(kR) I1(kr) / I1(kR)] / (2 pi)                 */
/*   3D  phi = [Q(r) - Q(R) J(kr) / J(kR)] / (4 pi r^2),                   */
/*       Q(r) = e^(-kr) (kr + 1),  J(t) = t cosh t - sinh t                 */
/* With the step's sample y = x + rho w, rho = R u2 (density 1 / (R |S|     */
/* rho^(d-1))), the weights are w_u = -|S| R rho^(d-1) G(rho) and w_g =     */
/* -|S| R rho^(d-1) phi(rho); at k -> 0 they are the Poisson weights of     */
/* orc_sphere_step.                                                         */
static double orc_j_cosh(double t) { /* t cosh t - sinh t */
  if (t < 0.1) {
    const double t2 = t * t;
    return t * t2 / 3.0 * (1.0 + t2 / 10.0 + t2 * t2 / 280.0 + t2 * t2 * t2 / 15120.0);
  }
  return t * cosh(t) - sinh(t);
}
void orc_screened_step_weights(int dim, double k, double R, double rho, double* wu, double* wg) {
  const double tr = k * rho, tR = k * R;
  if (dim == 2) {
    const double G = orc_bessel_k(0, tr) - orc_bessel_k(0, tR) * orc_bessel_i(0, tr) / orc_bessel_i(0, tR);
    const double phi = k * (orc_bessel_k(1, tr) - orc_bessel_k(1, tR) * orc_bessel_i(1, tr) / orc_bessel_i(1, tR));
    *wu = -R * rho * G;   /* 2 pi R rho x G / (2 pi) */
    *wg = -R * rho * phi;
  } else {
    *wu = -R * rho * sinh(tR - tr) / sinh(tR); /* 4 pi R rho^2 x G / (4 pi) */
    *wg = -R * (exp(-tr) * (tr + 1.0) - exp(-tR) * (tR + 1.0) * orc_j_cosh(tr) / orc_j_cosh(tR));
  }
}

/* The ball's screened Green's function seen from its centre, for a point at */
/* distance rho (0 < rho <= R): the Green's function of (sigma - Delta) on   */
/* B(x, R) that vanishes on the sphere (k = sqrt(sigma); see                 */
/* orc_screened_step_weights); k = 0 gives the Laplace ball's ln(R/rho)/(2   */
/* pi) (2D) and (1/rho - 1/R)/(4 pi) (3D).                                   */
double orc_ball_green_sigma(int dim, double k, double R, double rho) {
  if (!(k > 0.0))
    return dim == 2 ? log(R / rho) / (2.0 * ORC_PI) : (1.0 / rho - 1.0 / R) / (4.0 * ORC_PI);
  const double tr = k * rho, tR = k * R;
  if (dim == 2)
    return (orc_bessel_k(0, tr) - orc_bessel_k(0, tR) * orc_bessel_i(0, tr) / orc_bessel_i(0, tR)) / (2.0 * ORC_PI);
  if (tR > 20.0) /* sinh(a)/sinh(b) written with decaying exponentials */
    return exp(-tr) * (1.0 - exp(-2.0 * (tR - tr))) / ((1.0 - exp(-2.0 * tR)) * 4.0 * ORC_PI * rho);
  return sinh(tR - tr) / (4.0 * ORC_PI * rho * sinh(tR));
}

/* Throughput factor of a walk-on-stars step of the screened equation.  On a */
/* region St star-shaped about x inside B(x, R), Green's second identity     */
/* with the ball's Green's function G (above) gives u(x) as the integral of  */
/* u(z) (-dG/dn_z) over the parts of the boundary of St, plus the G-weighted */
/* Neumann and source terms.  G depends on r = |z - x| only, and a boundary  */
/* element seen from x under the solid angle dw has n_z . (z - x)/r dz =     */
/* r^(d-1) dw, so a direction drawn uniformly on the sphere (the walk's step) */
/* carries the factor W(r) = -|S| r^(d-1) G'(r) at the first boundary point  */
/* z it meets, r its distance:                                               */
/*   2D  W = kr [K1(kr) + K0(kR) I1(kr) / I0(kR)]                            */
/*   3D  W = [kr cosh(k(R - r)) + sinh(k(R - r))] / sinh(kR)                 */
/* W(R) is the screened mean-value factor of the ball and W -> 1 as r -> 0;  */
/* for k = 0 (Laplace) W = 1 for every r, the walk on stars of Sec. 3.1.     */
double orc_star_kernel_sigma(int dim, double k, double R, double r) {
  if (!(k > 0.0)) return 1.0;
  if (!(r > 0.0)) return 1.0;
  const double tr = k * r, tR = k * R;
  if (dim == 2)
    return tr * (orc_bessel_k(1, tr) + orc_bessel_k(0, tR) * orc_bessel_i(1, tr) / orc_bessel_i(0, tR));
  if (tR > 20.0)
    return exp(-tr) * (tr * (1.0 + exp(-2.0 * (tR - tr))) + (1.0 - exp(-2.0 * (tR - tr)))) / (1.0 - exp(-2.0 * tR));
  return (tr * cosh(tR - tr) + sinh(tR - tr)) / sinh(tR);
}

static void walk_one(const walk_ctx_t* w, const double* x0, uint64_t wid, double* U_out, double* grad_out,
                     int32_t* steps_out, int32_t* prim_out, double* pend_out, double* scale_out) {
  const int dim = w->bvh->m.dim;
  const int has_f = !fn_is_zero(w->f);
  double x[3] = {0, 0, 0}, pbar[3] = {0, 0, 0}, nu[3] = {0, 0, 0};
  for (int a = 0; a < dim; ++a) x[a] = x0[a];
  double usrc = 0.0, uabs = 0.0, wf0 = 0.0, wg0 = 0.0, R0 = 0.0, cv = 0.0;
  /* screened: throughput = product of the steps' factors C; the first     */
  /* step's C and gradient factor Qg (Sec. 3.1 with the screened ball)      */
  double thr = 1.0, C0 = 1.0, Qg0 = 1.0;
  int k = 0;
  int64_t prim = -1;
  for (;;) {
    const double d = sqrt(bvh_closest(w->bvh, x, pbar, &prim));
    ++k;
    if (k == 1) cv = g_at(w, pbar, prim);
    if (d < w->eps || k >= w->max_steps) break;
    const double R = d;
    const double thr_in = thr; /* throughput into this ball: weighs its source term */
    if (w->sqs > 0.0) {
      double Cs, Qs;
      orc_screened_factors(dim, w->sqs * R, &Cs, &Qs);
      thr *= Cs;
      if (k == 1) {
        C0 = Cs;
        Qg0 = Qs;
      }
    }
    double u[4];
    draw(w->seed, wid, (uint32_t)(k - 1), w->tag, u);
    double om[3] = {0, 0, 0}, rho, wu, wg;
    orc_sphere_step(dim, R, u[0], u[1], u[2], om, &rho, &wu, &wg);
    if (has_f) {
      if (w->sqs > 0.0) orc_screened_step_weights(dim, w->sqs, R, rho, &wu, &wg);
      double y[3] = {0, 0, 0};
      for (int a = 0; a < dim; ++a) y[a] = x[a] + rho * om[a];
      const double fy = orc_fn_eval(w->f, dim, y);
      usrc += thr_in * wu * fy;
      uabs += fabs(thr_in * wu * fy);
      if (k == 1) {
        wf0 = wu * fy;
        wg0 = wg * fy;
      }
    }
    if (k == 1) {
      R0 = R;
      for (int a = 0; a < dim; ++a) nu[a] = om[a];
    }
    for (int a = 0; a < dim; ++a) x[a] += R * om[a];
  }
  const double gend = g_at(w, pbar, prim);
  const double U = (k == 1 ? gend : thr * gend) + usrc;
  *U_out = U;
  /* magnitudes of the terms that form U and the gradient (test scaling only) */
  if (scale_out) {
    scale_out[0] = fabs(gend) + uabs;
    scale_out[1] = k == 1 ? 0.0 : ((double)dim / R0) * (fabs(gend) + uabs + fabs(wf0) + fabs(cv)) + fabs(wg0);
  }
  if (k == 1) {
    for (int a = 0; a < dim; ++a) grad_out[a] = 0.0;
  } else {
    /* screened: (U - wf0) / C0 estimates u at the first sphere point */
    const double s = w->sqs > 0.0 ? ((double)dim / R0) * Qg0 * ((U - wf0) / C0 - cv) + wg0
                                  : ((double)dim / R0) * (U - wf0 - cv) + wg0;
    for (int a = 0; a < dim; ++a) grad_out[a] = s * nu[a];
  }
  *steps_out = k;
  *prim_out = (int32_t)prim;
  if (pend_out)
    for (int a = 0; a < dim; ++a) pend_out[a] = pbar[a];
}

/* W walks from each of n start points; walk j of start i has id            */
/* id_base + i*W + j.  Outputs are per walk: U[n*W], grad[n*W*dim],         */
/* steps[n*W], prim[n*W], pend[n*W*dim] (pend may be NULL).                  */
void orc_walks_sigma(void* bvh, const double* g, const double* gv, const double* f, double sqs, const float* starts,
                     int64_t n, int32_t W, double eps, int32_t max_steps, uint64_t seed, uint64_t id_base, uint32_t tag,
                     double* U, double* grad, int32_t* steps, int32_t* prim, double* pend, double* scale) {
  walk_ctx_t w = {(const obvh_t*)bvh, g, f, eps, max_steps, seed, tag, gv, sqs};
  const int dim = w.bvh->m.dim;
  const int64_t total = n * (int64_t)W;
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t t = 0; t < total; ++t) {
    const int64_t i = t / W;
    double x0[3] = {0, 0, 0};
    for (int a = 0; a < dim; ++a) x0[a] = starts[i * dim + a];
    walk_one(&w, x0, id_base + (uint64_t)t, &U[t], &grad[t * dim], &steps[t], &prim[t],
             pend ? &pend[t * dim] : NULL, scale ? &scale[2 * t] : NULL);
  }
}

/* Poisson (sigma = 0) walks, g in closed form or from vertex values.       */
void orc_walks_vg(void* bvh, const double* g, const double* gv, const double* f, const float* starts, int64_t n,
                  int32_t W, double eps, int32_t max_steps, uint64_t seed, uint64_t id_base, uint32_t tag, double* U,
                  double* grad, int32_t* steps, int32_t* prim, double* pend, double* scale) {
  orc_walks_sigma(bvh, g, gv, f, 0.0, starts, n, W, eps, max_steps, seed, id_base, tag, U, grad, steps, prim, pend,
                  scale);
}

/* The same with closed-form boundary data g (no vertex values).           */
void orc_walks(void* bvh, const double* g, const double* f, const float* starts, int64_t n, int32_t W, double eps,
               int32_t max_steps, uint64_t seed, uint64_t id_base, uint32_t tag, double* U, double* grad,
               int32_t* steps, int32_t* prim, double* pend, double* scale) {
  orc_walks_vg(bvh, g, NULL, f, starts, n, W, eps, max_steps, seed, id_base, tag, U, grad, steps, prim, pend, scale);
}

/* ------------------------------------------------------------------------ */
/* Clamped double-layer kernel and its bias correction (Sec. 3.3, Eq. 8-9). */
/* The cache's u-term uses dG/dn clamped to [-c, c]; the remainder          */
/*   int [dG/dn - clamp(dG/dn)] u dz                                        */
/* is estimated per evaluation point x by importance sampling dG/dn dz,     */
/* the signed solid angle: a direction w uniform on the circle / sphere     */
/* (Philox id = point * n_dirs + j, word2 0, tag 4; 2D w = (cos 2 pi u0,    */
/* sin 2 pi u0); 3D z = 1 - 2 u0, phi = 2 pi u1) and every crossing z of   */
/* the ray x + t w (0 < t) with the sample surface contributes              */
/*   sign(n.w) (1 - c / |dG/dn(x, z)|) u(z) / n_dirs   when |dG/dn| > c,     */
/* |dG/dn| = |n.w| / (2 pi t) (2D), |n.w| / (4 pi t^2) (3D), so only t below */
/* 1/(2 pi c) or (4 pi c)^(-1/2) can matter.  The sample surface is the     */
/* mesh with each vertex moved by -l m_v (orc_offset_disp; l = 0: the mesh  */
/* itself), the surface the cache's samples lie on.  u(z)                   */
/* is estimated by W walks from z (FP32-rounded) on the domain's geometry   */
/* (tag 5, walk id = hit rank * W + j, hits ranked by point, direction and  */
/* distance along the ray).                                                  */
/* ------------------------------------------------------------------------ */
#define ORC_MAX_HITS 8
int orc_ray_hits(int dim, const float* V, const int32_t* F, int64_t np, double l, const double* mdisp,
                 const double* x, const double* om, double rmax, double* t_out, int64_t* e_out, double* nw_out) {
  int nh = 0;
  for (int64_t e = 0; e < np; ++e) {
    const int32_t* f = F + e * dim;
    double n[3] = {0, 0, 0};
    double P[3][3];
    for (int k = 0; k < dim; ++k)
      for (int a = 0; a < dim; ++a) P[k][a] = (double)V[dim * f[k] + a] - (mdisp ? l * mdisp[dim * f[k] + a] : 0.0);
    pts_measure_normal(dim, P, n);
    double t = -1.0;
    if (dim == 2) {
      double a[2], b[2];
      for (int k = 0; k < 2; ++k) {
        a[k] = P[0][k];
        b[k] = P[1][k];
      }
      const double ex = b[0] - a[0], ey = b[1] - a[1];
      const double den = om[0] * ey - om[1] * ex;
      if (fabs(den) < 1e-300) continue;
      const double ax = a[0] - x[0], ay = a[1] - x[1];
      const double tt = (ax * ey - ay * ex) / den;
      const double ss = (ax * om[1] - ay * om[0]) / den;
      if (ss < 0.0 || ss > 1.0) continue;
      t = tt;
    } else {
      double a[3], b[3], c[3];
      for (int k = 0; k < 3; ++k) {
        a[k] = P[0][k];
        b[k] = P[1][k];
        c[k] = P[2][k];
      }
      /* Moller-Trumbore (J. Graphics Tools 2(1), 1997) */
      double e1[3], e2[3], tv[3];
      for (int k = 0; k < 3; ++k) {
        e1[k] = b[k] - a[k];
        e2[k] = c[k] - a[k];
        tv[k] = x[k] - a[k];
      }
      const double pv[3] = {om[1] * e2[2] - om[2] * e2[1], om[2] * e2[0] - om[0] * e2[2],
                            om[0] * e2[1] - om[1] * e2[0]};
      const double det = dot3d(e1, pv);
      if (fabs(det) < 1e-300) continue;
      const double u = dot3d(tv, pv) / det;
      if (u < 0.0 || u > 1.0) continue;
      const double qv[3] = {tv[1] * e1[2] - tv[2] * e1[1], tv[2] * e1[0] - tv[0] * e1[2],
                            tv[0] * e1[1] - tv[1] * e1[0]};
      const double v = dot3d(om, qv) / det;
      if (v < 0.0 || u + v > 1.0) continue;
      t = dot3d(e2, qv) / det;
    }
    if (!(t > 0.0) || t > rmax) continue;
    double nw = 0.0;
    for (int k = 0; k < dim; ++k) nw += n[k] * om[k];
    /* insert sorted by t (ties by element), keep the nearest ORC_MAX_HITS */
    int pos = nh;
    while (pos > 0 && (t_out[pos - 1] > t || (t_out[pos - 1] == t && e_out[pos - 1] > e))) --pos;
    if (pos >= ORC_MAX_HITS) continue;
    const int last = nh < ORC_MAX_HITS ? nh : ORC_MAX_HITS - 1;
    for (int q = last; q > pos; --q) {
      t_out[q] = t_out[q - 1];
      e_out[q] = e_out[q - 1];
      nw_out[q] = nw_out[q - 1];
    }
    t_out[pos] = t;
    e_out[pos] = e;
    nw_out[pos] = nw;
    if (nh < ORC_MAX_HITS) ++nh;
  }
  return nh;
}

static void unit_direction(int dim, const double* u, double* om) {
  if (dim == 2) {
    om[0] = cos(2.0 * ORC_PI * u[0]);
    om[1] = sin(2.0 * ORC_PI * u[0]);
  } else {
    const double zc = 1.0 - 2.0 * u[0], phi = 2.0 * ORC_PI * u[1];
    const double s = sqrt(fmax(0.0, 1.0 - zc * zc));
    om[0] = s * cos(phi);
    om[1] = s * sin(phi);
    om[2] = zc;
  }
}

/* u_corr[m] (overwritten) and the number of contributing hits. */
int64_t orc_clamp_correction(void* bvh, const double* g, const double* gv, double sqs, const float* Vs,
                             const int32_t* Fs, int64_t nps, double l, const double* pts, int64_t m, double c,
                             int32_t n_dirs, int32_t W, double eps, int32_t max_steps, uint64_t seed,
                             double* u_corr) {
  const obvh_t* B = (const obvh_t*)bvh;
  const int dim = B->m.dim;
  const double rmax = dim == 2 ? 1.0 / (2.0 * ORC_PI * c) : sqrt(1.0 / (4.0 * ORC_PI * c));
  const int64_t slots = m * (int64_t)n_dirs * ORC_MAX_HITS;
  int64_t nvs = 0;
  for (int64_t i = 0; i < nps * dim; ++i)
    if (Fs[i] + 1 > nvs) nvs = Fs[i] + 1;
  double* mdisp = (double*)malloc(sizeof(double) * (size_t)nvs * dim);
  orc_offset_disp(dim, Vs, nvs, Fs, nps, NULL, mdisp);
  double* hz = (double*)malloc((size_t)slots * 3 * sizeof(double));
  double* hw = (double*)malloc((size_t)slots * sizeof(double));
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t q = 0; q < m * (int64_t)n_dirs; ++q) {
    const int64_t p = q / n_dirs;
    double u[4], om[3] = {0, 0, 0};
    draw(seed, (uint64_t)q, 0u, 4u, u);
    unit_direction(dim, u, om);
    double t[ORC_MAX_HITS], nw[ORC_MAX_HITS];
    int64_t e[ORC_MAX_HITS];
    const int nh = orc_ray_hits(dim, Vs, Fs, nps, l, mdisp, pts + p * dim, om, rmax, t, e, nw);
    for (int k = 0; k < ORC_MAX_HITS; ++k) {
      const int64_t sl = q * ORC_MAX_HITS + k;
      hw[sl] = 0.0;
      if (k >= nh) continue;
      const double gn = dim == 2 ? fabs(nw[k]) / (2.0 * ORC_PI * t[k]) : fabs(nw[k]) / (4.0 * ORC_PI * t[k] * t[k]);
      if (!(gn > c)) continue;
      hw[sl] = (nw[k] > 0.0 ? 1.0 : -1.0) * (1.0 - c / gn) / n_dirs;
      for (int a = 0; a < dim; ++a) hz[3 * sl + a] = (double)(float)(pts[p * dim + a] + t[k] * om[a]);
    }
  }
  /* rank the contributing hits in slot order */
  int64_t nhit = 0;
  int64_t* rank = (int64_t*)malloc((size_t)slots * sizeof(int64_t));
  for (int64_t sl = 0; sl < slots; ++sl) rank[sl] = hw[sl] != 0.0 ? nhit++ : -1;
  for (int64_t p = 0; p < m; ++p) u_corr[p] = 0.0;
  walk_ctx_t w = {B, g, NULL, eps, max_steps, seed, 5u, gv, sqs};
  double* contrib = (double*)calloc((size_t)slots, sizeof(double));
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t sl = 0; sl < slots; ++sl) {
    if (rank[sl] < 0) continue;
    double sum = 0.0;
    for (int32_t j = 0; j < W; ++j) {
      double U, grad[3];
      int32_t steps, prim;
      walk_one(&w, hz + 3 * sl, (uint64_t)rank[sl] * W + j, &U, grad, &steps, &prim, NULL, NULL);
      sum += U;
    }
    contrib[sl] = hw[sl] * sum / W;
  }
  for (int64_t sl = 0; sl < slots; ++sl) u_corr[sl / ((int64_t)n_dirs * ORC_MAX_HITS)] += contrib[sl];
  free(contrib);
  free(rank);
  free(hz);
  free(hw);
  free(mdisp);
  return nhit;
}

/* Per-sample means over the W walks of each start (Alg. 1: the pointwise   */
/* estimates u^ and du/dn^ of a boundary sample).  du/dn^ = n . grad.        */
void orc_reduce_walks(int dim, int64_t n, int32_t W, const double* U, const double* grad, const float* nrm,
                      double* u_hat, double* q_hat) {
  for (int64_t i = 0; i < n; ++i) {
    double su = 0.0, sq = 0.0;
    for (int32_t j = 0; j < W; ++j) {
      const int64_t t = i * W + j;
      su += U[t];
      if (nrm) {
        double g = 0.0;
        for (int a = 0; a < dim; ++a) g += (double)nrm[i * dim + a] * grad[t * dim + a];
        sq += g;
      }
    }
    u_hat[i] = su / W;
    if (q_hat) q_hat[i] = sq / W;
  }
}

/* ------------------------------------------------------------------------ */
/* Source samples (Sec. 4 "Sampling", Alg. 1 y ~ p^R): a jittered grid of   */
/* G0 x G1 cells over the boundary's bounding box; candidate c draws        */
/* (u0,u1) from Philox (id = c, word2 = 0, tag = 2); kept when the canonical */
/* FP32 crossing test puts it inside.  With p = 1/|box| on the box and the  */
/* indicator of the domain, the weight of a kept sample is f(y) |box| and    */
/* the source estimator divides by the number of candidates G0*G1.          */
/* Kept samples are returned in candidate order.  The region the BIE of the */
/* cache refers to is the one inside the offset boundary (Sec. 3.2), so the */
/* inside test takes the moved vertices Vin (orc_offset_vertices; NULL =   */
/* V itself, offset 0); the box stays the boundary's own.                   */
/* ------------------------------------------------------------------------ */
int64_t orc_sample_source2d(const float* V, int64_t nv, const int32_t* F, int64_t np, int32_t G0, int32_t G1,
                            uint64_t seed, const double* f, const float* Vin, float* y_out, double* c_out) {
  float lo[2] = {INFINITY, INFINITY}, hi[2] = {-INFINITY, -INFINITY};
  for (int64_t i = 0; i < nv; ++i)
    for (int a = 0; a < 2; ++a) {
      if (V[2 * i + a] < lo[a]) lo[a] = V[2 * i + a];
      if (V[2 * i + a] > hi[a]) hi[a] = V[2 * i + a];
    }
  const double ext0 = (double)hi[0] - (double)lo[0], ext1 = (double)hi[1] - (double)lo[1];
  const double area = ext0 * ext1;
  const int64_t ncand = (int64_t)G0 * G1;
  int64_t kept = 0;
  for (int64_t c = 0; c < ncand; ++c) {
    double u[4];
    draw(seed, (uint64_t)c, 0u, 2u, u);
    const int64_t c0 = c % G0, c1 = c / G0;
    const double y0 = (double)lo[0] + ((double)c0 + u[0]) * (ext0 / G0);
    const double y1 = (double)lo[1] + ((double)c1 + u[1]) * (ext1 / G1);
    const float fy0 = (float)y0, fy1 = (float)y1;
    if (!inside2d_f32(Vin ? Vin : V, F, np, fy0, fy1)) continue;
    const double yy[2] = {fy0, fy1};
    y_out[2 * kept] = fy0;
    y_out[2 * kept + 1] = fy1;
    c_out[kept] = orc_fn_eval(f, 2, yy) * area;
    ++kept;
  }
  return kept;
}

/* ------------------------------------------------------------------------ */
/* Generalized winding number of a triangle mesh at p (Jacobson, Kavan and  */
/* Sorkine-Hornung, SIGGRAPH 2013): the sum of the signed solid angles of   */
/* its triangles seen from p over 4 pi.  The solid angle of triangle        */
/* (a, b, c) relative to p is 2 atan2(A . (B x C), |A||B||C| + (A.B)|C|     */
/* + (A.C)|B| + (B.C)|A|) with A = a - p, ... (Van Oosterom and Strackee,   */
/* IEEE TBME 1983).  It is 1 inside a closed outward-wound surface, 0       */
/* outside, and counts nested or overlapping shells with their orientation, */
/* which is how an unrepaired self-intersecting boundary is classified.     */
/* ------------------------------------------------------------------------ */
double orc_winding3d(const float* V, const int32_t* F, int64_t np, const double* p) {
  double w = 0.0;
  for (int64_t e = 0; e < np; ++e) {
    double A[3], B[3], Cc[3];
    for (int a = 0; a < 3; ++a) {
      A[a] = (double)V[3 * (int64_t)F[3 * e] + a] - p[a];
      B[a] = (double)V[3 * (int64_t)F[3 * e + 1] + a] - p[a];
      Cc[a] = (double)V[3 * (int64_t)F[3 * e + 2] + a] - p[a];
    }
    const double la = sqrt(dot3d(A, A)), lb = sqrt(dot3d(B, B)), lc = sqrt(dot3d(Cc, Cc));
    const double bxc[3] = {B[1] * Cc[2] - B[2] * Cc[1], B[2] * Cc[0] - B[0] * Cc[2], B[0] * Cc[1] - B[1] * Cc[0]};
    const double num = dot3d(A, bxc);
    const double den = la * lb * lc + dot3d(A, B) * lc + dot3d(A, Cc) * lb + dot3d(B, Cc) * la;
    w += 2.0 * atan2(num, den);
  }
  return w / (4.0 * ORC_PI);
}

/* Source samples in 3D (Sec. 4 "Sampling"): a jittered grid of G0 x G1 x  */
/* G2 cells over the bounding box; candidate c (cell c0 = c mod G0,         */
/* c1 = (c / G0) mod G1, c2 = c / (G0 G1)) draws (u0,u1,u2) from Philox      */
/* (id = c, word2 = 0, tag = 2) and is kept when the winding number is      */
/* above 1/2 (winding number of the moved mesh Vin, as in 2D; NULL = V).   */
/* Weight f(y) |box|; the estimator divides by G0 G1 G2.                    */
/* winding_out (may be NULL) receives every candidate's winding number.     */
int64_t orc_sample_source3d(const float* V, int64_t nv, const int32_t* F, int64_t np, int32_t G0, int32_t G1,
                            int32_t G2, uint64_t seed, const double* f, const float* Vin, float* y_out, double* c_out,
                            double* winding_out) {
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t i = 0; i < nv; ++i)
    for (int a = 0; a < 3; ++a) {
      if (V[3 * i + a] < lo[a]) lo[a] = V[3 * i + a];
      if (V[3 * i + a] > hi[a]) hi[a] = V[3 * i + a];
    }
  const double ext[3] = {(double)hi[0] - lo[0], (double)hi[1] - lo[1], (double)hi[2] - lo[2]};
  const int32_t G[3] = {G0, G1, G2};
  const double vol = ext[0] * ext[1] * ext[2];
  const int64_t ncand = (int64_t)G0 * G1 * G2;
  float* yc = (float*)malloc((size_t)ncand * 3 * sizeof(float));
  uint8_t* keep = (uint8_t*)malloc((size_t)ncand);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t c = 0; c < ncand; ++c) {
    double u[4];
    draw(seed, (uint64_t)c, 0u, 2u, u);
    const int64_t ci[3] = {c % G0, (c / G0) % G1, c / ((int64_t)G0 * G1)};
    double y[3];
    for (int a = 0; a < 3; ++a) {
      yc[3 * c + a] = (float)((double)lo[a] + ((double)ci[a] + u[a]) * (ext[a] / G[a]));
      y[a] = yc[3 * c + a];
    }
    const double w = orc_winding3d(Vin ? Vin : V, F, np, y);
    if (winding_out) winding_out[c] = w;
    keep[c] = w > 0.5;
  }
  int64_t kept = 0;
  for (int64_t c = 0; c < ncand; ++c) {
    if (!keep[c]) continue;
    double y[3];
    for (int a = 0; a < 3; ++a) {
      y_out[3 * kept + a] = yc[3 * c + a];
      y[a] = yc[3 * c + a];
    }
    c_out[kept] = orc_fn_eval(f, 3, y) * vol;
    ++kept;
  }
  free(yc);
  free(keep);
  return kept;
}

/* ------------------------------------------------------------------------ */
/* The gather: Eq. 3-6 and the splat loops of Alg. 1, as a direct double    */
/* loop.  For every evaluation point x and boundary sample (z, n, u^, q^):  */
/*   u_bnd    += (dG/dn(x,z) u^ - G(x,z) q^) / p,        p = 1/|dOmega|      */
/*   grad_bnd += (d2G/dxdn(x,z) u^ - dG/dx(x,z) q^) / p                      */
/* and for every source sample (y, c = f(y)/p^Omega):                        */
/*   u_src    += G(x,y) c,    grad_src += dG/dx(x,y) c                       */
/* Returns SUMS (Alg. 1 running sums); the caller divides by N and M.       */
/* jac (may be NULL = all 1): per boundary sample, 1/p = |dOmega| jac       */
/* (samples on the offset boundary, see sample_boundary).                   */
/* ------------------------------------------------------------------------ */
/* clamp_c > 0: dG/dn in the u term clamped to [-c, c] (Sec. 3.3, Eq. 9);  */
/* the gradient terms are not clamped.                                       */
void orc_gather_full(int dim, double sqs, double clamp_c, int64_t N, const double* z, const double* nz,
                     const double* u_hat, const double* q_hat, double bnd_measure, const double* jac, int64_t Ms,
                     const double* y,
                     const double* c, int64_t M, const double* x, double* u_bnd, double* u_src, double* g_bnd,
                     double* g_src, double* abs_out) {
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t k = 0; k < M; ++k) {
    double xk[3] = {0, 0, 0}, zz[3] = {0, 0, 0}, nn[3] = {0, 0, 0}, G[8];
    for (int a = 0; a < dim; ++a) xk[a] = x[k * dim + a];
    double ub = 0.0, us = 0.0, gb[3] = {0, 0, 0}, gs[3] = {0, 0, 0};
    /* sums of |term| (test scaling only): [u_bnd, g_bnd(dim), u_src, g_src(dim)] */
    double ab[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t i = 0; i < N; ++i) {
      for (int a = 0; a < dim; ++a) {
        zz[a] = z[i * dim + a];
        nn[a] = nz[i * dim + a];
      }
      orc_green_sigma(dim, sqs, xk, zz, nn, G);
      const double dGdn = clamp_c > 0.0 ? fmax(-clamp_c, fmin(clamp_c, G[1 + dim])) : G[1 + dim];
      const double ip = jac ? bnd_measure * jac[i] : bnd_measure; /* 1/p of sample i */
      const double tu = (dGdn * u_hat[i] - G[0] * q_hat[i]) * ip;
      ub += tu;
      ab[0] += fabs(tu);
      for (int a = 0; a < dim; ++a) {
        const double tg = (G[2 + dim + a] * u_hat[i] - G[1 + a] * q_hat[i]) * ip;
        gb[a] += tg;
        ab[1 + a] += fabs(tg);
      }
    }
    for (int64_t j = 0; j < Ms; ++j) {
      for (int a = 0; a < dim; ++a) zz[a] = y[j * dim + a];
      orc_green_sigma(dim, sqs, xk, zz, nn, G);
      us += G[0] * c[j];
      ab[1 + dim] += fabs(G[0] * c[j]);
      for (int a = 0; a < dim; ++a) {
        gs[a] += G[1 + a] * c[j];
        ab[2 + dim + a] += fabs(G[1 + a] * c[j]);
      }
    }
    u_bnd[k] = ub;
    u_src[k] = us;
    if (abs_out)
      for (int q = 0; q < 2 + 2 * dim; ++q) abs_out[k * (2 + 2 * dim) + q] = ab[q];
    for (int a = 0; a < dim; ++a) {
      if (g_bnd) g_bnd[k * dim + a] = gb[a];
      if (g_src) g_src[k * dim + a] = gs[a];
    }
  }
}

void orc_gather_sigma(int dim, double sqs, int64_t N, const double* z, const double* nz, const double* u_hat,
                      const double* q_hat, double bnd_measure, int64_t Ms, const double* y, const double* c, int64_t M,
                      const double* x, double* u_bnd, double* u_src, double* g_bnd, double* g_src, double* abs_out) {
  orc_gather_full(dim, sqs, 0.0, N, z, nz, u_hat, q_hat, bnd_measure, NULL, Ms, y, c, M, x, u_bnd, u_src, g_bnd,
                  g_src, abs_out);
}

void orc_gather(int dim, int64_t N, const double* z, const double* nz, const double* u_hat, const double* q_hat,
                double bnd_measure, int64_t Ms, const double* y, const double* c, int64_t M, const double* x,
                double* u_bnd, double* u_src, double* g_bnd, double* g_src, double* abs_out) {
  orc_gather_full(dim, 0.0, 0.0, N, z, nz, u_hat, q_hat, bnd_measure, NULL, Ms, y, c, M, x, u_bnd, u_src, g_bnd,
                  g_src, abs_out);
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Threads of later parallel loops (timing the oracle on one core). */
void orc_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* ------------------------------------------------------------------------ */
/* Walk on stars (Sec. 3.1; Fig. "WoS vs WoSt") for a mixed boundary:       */
/* Laplace(u) = f in Omega, u = g on the Dirichlet part, du/dn = h on the   */
/* Neumann part (Eq. 1 with sigma = 0).                                     */
/*                                                                          */
/* Step at x: d_D = distance to the Dirichlet part; the walk stops when     */
/* d_D < eps and returns g at the closest Dirichlet point.  Otherwise the   */
/* star radius is R = max(min(d_D, d_sil), eps), d_sil the distance to the  */
/* closest silhouette point of the Neumann part seen from x, so that every  */
/* ray from x crosses the Neumann part at most once inside B(x, R).  A      */
/* direction w is drawn uniformly (on the inward hemisphere when x lies on  */
/* the Neumann part); the ray x + t w, 0 < t <= R, is intersected with the  */
/* Neumann part; the walk moves to the first hit (and is then on the        */
/* boundary with that element's normal) or to x + R w.  With the ball's    */
/* Green's function of -Laplacian, G^B(t) = ln(R/t)/(2 pi) (2D),            */
/* (1/t - 1/R)/(4 pi) (3D), Green's second identity on the star region     */
/*   a(x) u(x) = int_{dSt} u dG^B/dn  -  int_St G^B f  +  int_{dSt_N} G^B h  */
/* (a = 1 inside, 1/2 on a smooth boundary point; the first integral is    */
/* the solid angle measure / |S|) gives per step, with r = min(t_hit, R):   */
/*   source  y = x + rho w, rho = r u2:                                      */
/*           w_u = -r rho ln(R/rho) (2D),  -r rho (1 - rho/R) (3D)           */
/*   Neumann term: a point z on the Neumann part inside B(x, R), chosen by  */
/*           measure among the Neumann elements that reach into the ball    */
/*           (total measure A) and uniformly on the element, adds           */
/*           (1/a) G^B(|z - x|) h(z) A when z is inside the ball and seen   */
/*           from x (no Neumann crossing between, elements within 1e-4 of   */
/*           parallel to the sight line not counting), else nothing;        */
/*           a = 1/2 on the boundary.  Draws: Philox (walk id, step - 1, tag + 8):   */
/*           u0 picks the element (cumulative measure in element order),    */
/*           u1, u2 the point (as the boundary sampler places points).      */
/*           For an x on the Neumann part the element under x is left out  */
/*           of this choice and sampled around x instead (wost_own_term).   */
/*   U = g(end) + sum w_u f(y) + sum of the Neumann terms.                   */
/* A walk that starts inside the domain takes its first step in the ball of */
/* radius d_all (distance to the whole boundary, no Neumann part inside)    */
/* and estimates the gradient there as the walk on spheres does (Eq. 7);   */
/* when d_all < eps the first step is a star step and the gradient is 0.    */
/* Draws: Philox (id = walk id, word2 = step - 1, tag), w from (u0, u1) as  */
/* on the sphere and flipped to -w when it points out of an on-boundary x,  */
/* rho from u2.                                                              */
/*                                                                          */
/* Silhouettes: a Neumann vertex (2D) or edge (3D) shared by two Neumann    */
/* elements with outward normals n0, n1; with a = (vertex or the edge's     */
/* first vertex) - x and d_k = n_k . a, treated as zero when |d_k| <= tau,  */
/* it is a silhouette when one d_k is zero and the other negative (the      */
/* element seen edge-on, its neighbour facing away: a reflex vertex or      */
/* edge) or both are non-zero with opposite signs.  Vertices or edges with one or more than two        */
/* Neumann elements and no Dirichlet element are always silhouettes; those  */
/* touching a Dirichlet element are skipped (never closer than d_D).        */
/* tau = 2^-18 x the bounding-box diagonal.  All queries are brute force.   */
/* ------------------------------------------------------------------------ */
typedef struct {
  int dim;
  int64_t np, nv;
  double* V;          /* [nv][dim] */
  int32_t* F;         /* [np][dim] */
  uint8_t* neu;       /* [np] */
  double* nrm;        /* [np][dim] outward normals */
  double* meas;       /* [np] element measures */
  void* all;          /* BVH of the whole boundary */
  void* dir;          /* BVH of the Dirichlet elements */
  int64_t* dir_ids;   /* Dirichlet BVH element -> whole element */
  int64_t n_neu;
  int64_t* neu_ids;   /* Neumann elements (whole numbering, increasing) */
  int64_t n_sil;
  double* sil;        /* per candidate: 2D [v(2) n0(2) n1(2) always], 3D [a(3) b(3) n0(3) n1(3) always] */
  double tau;
  double diag;        /* bounding-box diagonal */
} wost_t;

static int sil_stride(int dim) { return dim == 2 ? 7 : 13; }

typedef struct {
  int32_t lo, hi, e;
} edge_ref_t;

static int cmp_edge(const void* x, const void* y) {
  const edge_ref_t* a = (const edge_ref_t*)x;
  const edge_ref_t* b = (const edge_ref_t*)y;
  if (a->lo != b->lo) return a->lo < b->lo ? -1 : 1;
  if (a->hi != b->hi) return a->hi < b->hi ? -1 : 1;
  return (a->e > b->e) - (a->e < b->e);
}

void* orc_wost_create(int dim, const float* V, int64_t nv, const int32_t* F, int64_t np, const uint8_t* neu) {
  wost_t* w = (wost_t*)calloc(1, sizeof(wost_t));
  w->dim = dim;
  w->np = np;
  w->nv = nv;
  w->V = (double*)malloc(sizeof(double) * nv * dim);
  for (int64_t i = 0; i < nv * dim; ++i) w->V[i] = V[i];
  w->F = (int32_t*)malloc(sizeof(int32_t) * np * dim);
  memcpy(w->F, F, sizeof(int32_t) * np * dim);
  w->neu = (uint8_t*)malloc((size_t)np);
  memcpy(w->neu, neu, (size_t)np);
  w->nrm = (double*)malloc(sizeof(double) * np * dim);
  w->meas = (double*)malloc(sizeof(double) * np);
  for (int64_t e = 0; e < np; ++e) w->meas[e] = elem_measure_normal(dim, V, F + e * dim, w->nrm + e * dim);
  w->all = orc_bvh_create(dim, V, nv, F, np);
  int64_t nd = 0;
  for (int64_t e = 0; e < np; ++e) nd += neu[e] ? 0 : 1;
  int32_t* FD = (int32_t*)malloc(sizeof(int32_t) * (nd > 0 ? nd : 1) * dim);
  w->dir_ids = (int64_t*)malloc(sizeof(int64_t) * (nd > 0 ? nd : 1));
  w->neu_ids = (int64_t*)malloc(sizeof(int64_t) * (np - nd > 0 ? np - nd : 1));
  int64_t q = 0;
  for (int64_t e = 0; e < np; ++e) {
    if (neu[e]) {
      w->neu_ids[w->n_neu++] = e;
    } else {
      memcpy(FD + q * dim, F + e * dim, sizeof(int32_t) * dim);
      w->dir_ids[q++] = e;
    }
  }
  w->dir = orc_bvh_create(dim, V, nv, FD, nd);
  free(FD);
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t i = 0; i < nv; ++i)
    for (int a = 0; a < dim; ++a) {
      if (V[i * dim + a] < lo[a]) lo[a] = V[i * dim + a];
      if (V[i * dim + a] > hi[a]) hi[a] = V[i * dim + a];
    }
  double diag = 0.0;
  for (int a = 0; a < dim; ++a) diag += (hi[a] - lo[a]) * (hi[a] - lo[a]);
  w->tau = ldexp(1.0, -18) * (diag > 0.0 ? sqrt(diag) : 1.0);
  w->diag = sqrt(diag);
  /* silhouette candidates from the elements around each vertex (2D) or    */
  /* edge (3D)                                                              */
  const int ss = sil_stride(dim);
  if (dim == 2) {
    int64_t* cnt_n = (int64_t*)calloc((size_t)nv, sizeof(int64_t));
    int64_t* cnt_d = (int64_t*)calloc((size_t)nv, sizeof(int64_t));
    int64_t* first = (int64_t*)malloc(sizeof(int64_t) * nv);
    int64_t* second = (int64_t*)malloc(sizeof(int64_t) * nv);
    for (int64_t v = 0; v < nv; ++v) first[v] = second[v] = -1;
    for (int64_t e = 0; e < np; ++e)
      for (int k = 0; k < 2; ++k) {
        const int32_t v = F[2 * e + k];
        if (!neu[e]) {
          ++cnt_d[v];
        } else {
          if (cnt_n[v] == 0) first[v] = e;
          if (cnt_n[v] == 1) second[v] = e;
          ++cnt_n[v];
        }
      }
    w->sil = (double*)malloc(sizeof(double) * ss * (nv > 0 ? nv : 1));
    for (int64_t v = 0; v < nv; ++v) {
      if (cnt_n[v] == 0 || cnt_d[v] > 0) continue;
      double* c = w->sil + w->n_sil * ss;
      c[0] = w->V[2 * v];
      c[1] = w->V[2 * v + 1];
      if (cnt_n[v] == 2) {
        for (int a = 0; a < 2; ++a) {
          c[2 + a] = w->nrm[2 * first[v] + a];
          c[4 + a] = w->nrm[2 * second[v] + a];
        }
        c[6] = 0.0;
      } else {
        for (int a = 0; a < 4; ++a) c[2 + a] = 0.0;
        c[6] = 1.0;
      }
      ++w->n_sil;
    }
    free(cnt_n);
    free(cnt_d);
    free(first);
    free(second);
  } else {
    edge_ref_t* ed = (edge_ref_t*)malloc(sizeof(edge_ref_t) * 3 * (np > 0 ? np : 1));
    for (int64_t e = 0; e < np; ++e)
      for (int k = 0; k < 3; ++k) {
        const int32_t a = F[3 * e + k], b = F[3 * e + (k + 1) % 3];
        ed[3 * e + k].lo = a < b ? a : b;
        ed[3 * e + k].hi = a < b ? b : a;
        ed[3 * e + k].e = (int32_t)e;
      }
    qsort(ed, (size_t)(3 * np), sizeof(edge_ref_t), cmp_edge);
    w->sil = (double*)malloc(sizeof(double) * ss * (3 * np > 0 ? 3 * np : 1));
    for (int64_t i = 0; i < 3 * np;) {
      int64_t j = i;
      int n_n = 0, n_d = 0;
      int32_t en[2] = {-1, -1};
      while (j < 3 * np && ed[j].lo == ed[i].lo && ed[j].hi == ed[i].hi) {
        if (neu[ed[j].e]) {
          if (n_n < 2) en[n_n] = ed[j].e;
          ++n_n;
        } else {
          ++n_d;
        }
        ++j;
      }
      if (n_n > 0 && n_d == 0) {
        double* c = w->sil + w->n_sil * ss;
        for (int a = 0; a < 3; ++a) {
          c[a] = w->V[3 * (int64_t)ed[i].lo + a];
          c[3 + a] = w->V[3 * (int64_t)ed[i].hi + a];
        }
        if (n_n == 2) {
          for (int a = 0; a < 3; ++a) {
            c[6 + a] = w->nrm[3 * (int64_t)en[0] + a];
            c[9 + a] = w->nrm[3 * (int64_t)en[1] + a];
          }
          c[12] = 0.0;
        } else {
          for (int a = 0; a < 6; ++a) c[6 + a] = 0.0;
          c[12] = 1.0;
        }
        ++w->n_sil;
      }
      i = j;
    }
    free(ed);
  }
  return w;
}

void orc_wost_free(void* h) {
  wost_t* w = (wost_t*)h;
  if (!w) return;
  orc_bvh_free(w->all);
  orc_bvh_free(w->dir);
  free(w->V);
  free(w->F);
  free(w->neu);
  free(w->nrm);
  free(w->meas);
  free(w->dir_ids);
  free(w->neu_ids);
  free(w->sil);
  free(w);
}

int64_t orc_wost_counts(void* h, int64_t* out) {
  const wost_t* w = (const wost_t*)h;
  out[0] = w->np - w->n_neu;
  out[1] = w->n_neu;
  out[2] = w->n_sil;
  return w->n_sil;
}

/* Distance from x to the closest silhouette point (INFINITY if none). */
static double wost_sil_dist(const wost_t* w, const double* x) {
  const int dim = w->dim, ss = sil_stride(dim);
  double best = INFINITY;
  for (int64_t i = 0; i < w->n_sil; ++i) {
    const double* c = w->sil + i * ss;
    double a[3] = {0, 0, 0};
    for (int k = 0; k < dim; ++k) a[k] = c[k] - x[k];
    const int always = c[dim == 2 ? 6 : 12] != 0.0;
    int is_sil = always;
    if (!always) {
      const double* n0 = c + (dim == 2 ? 2 : 6);
      const double* n1 = c + (dim == 2 ? 4 : 9);
      double d0 = 0.0, d1 = 0.0;
      for (int k = 0; k < dim; ++k) {
        d0 += n0[k] * a[k];
        d1 += n1[k] * a[k];
      }
      const int z0 = fabs(d0) <= w->tau, z1 = fabs(d1) <= w->tau;
      /* one element edge-on (zero): a silhouette when the other faces away */
      is_sil = (z0 && !z1 && d1 < 0.0) || (z1 && !z0 && d0 < 0.0) || (!z0 && !z1 && ((d0 > 0.0) != (d1 > 0.0)));
    }
    if (!is_sil) continue;
    double d2;
    if (dim == 2) {
      d2 = a[0] * a[0] + a[1] * a[1];
    } else {
      double cp[3];
      const double b[3] = {c[3], c[4], c[5]};
      d2 = seg3_closest64(c, b, x, cp);
    }
    if (d2 < best) best = d2;
  }
  return sqrt(best);
}

/* First crossing of the ray x + t w, 0 < t <= tmax, with the Neumann part,  */
/* skipping element `skip` (whole numbering, -1 for none); ties go to the    */
/* lowest element.  Returns the element (or -1) and sets *t_out.             */
static int ray_elem(const wost_t* w, int64_t e, const double* x, const double* om, double* t_out) {
  const int dim = w->dim;
  *t_out = -INFINITY;
  const int32_t* f = w->F + e * dim;
  double t;
  if (dim == 2) {
    const double* a = w->V + 2 * (int64_t)f[0];
    const double* b = w->V + 2 * (int64_t)f[1];
    const double abx = b[0] - a[0], aby = b[1] - a[1];
    const double den = om[0] * aby - om[1] * abx;
    if (den == 0.0) return 0;
    const double qx = a[0] - x[0], qy = a[1] - x[1];
    const double s = (qx * om[1] - qy * om[0]) / den;
    if (s < 0.0 || s > 1.0) return 0;
    t = (qx * aby - qy * abx) / den;
  } else {
    /* Moller-Trumbore (J. Graphics Tools 2(1), 1997) */
    const double* a = w->V + 3 * (int64_t)f[0];
    const double* b = w->V + 3 * (int64_t)f[1];
    const double* c = w->V + 3 * (int64_t)f[2];
    double e1[3], e2[3], P[3], T[3], Q[3];
    for (int k = 0; k < 3; ++k) {
      e1[k] = b[k] - a[k];
      e2[k] = c[k] - a[k];
      T[k] = x[k] - a[k];
    }
    P[0] = om[1] * e2[2] - om[2] * e2[1];
    P[1] = om[2] * e2[0] - om[0] * e2[2];
    P[2] = om[0] * e2[1] - om[1] * e2[0];
    const double det = dot3d(e1, P);
    if (det == 0.0) return 0;
    const double u = dot3d(T, P) / det;
    if (u < 0.0 || u > 1.0) return 0;
    Q[0] = T[1] * e1[2] - T[2] * e1[1];
    Q[1] = T[2] * e1[0] - T[0] * e1[2];
    Q[2] = T[0] * e1[1] - T[1] * e1[0];
    const double v = dot3d(om, Q) / det;
    if (v < 0.0 || u + v > 1.0) return 0;
    t = dot3d(e2, Q) / det;
  }
  *t_out = t;
  return t > 0.0;
}
/* (ray_elem sets *t_out whenever the line meets the element; it returns 1 */
/* only for t > 0.)                                                         */

/* Only elements the ray leaves the domain through (n . w > 0) count: a ray */
/* from inside meets such a front face first, and a walker on an edge       */
/* between two Neumann elements is not stopped by the one it moves away     */
/* from.  Crossings with t in (-tau, 0] count as crossings at t = 0: that   */
/* walker, looking out through the other element, does not pass it.        */
static int64_t wost_ray(const wost_t* w, const double* x, const double* om, double tmax, int64_t skip,
                        double* t_out) {
  double best = INFINITY;
  int64_t be = -1;
  for (int64_t q = 0; q < w->n_neu; ++q) {
    const int64_t e = w->neu_ids[q];
    double t, cs = 0.0;
    if (e == skip) continue;
    for (int a = 0; a < w->dim; ++a) cs += w->nrm[e * w->dim + a] * om[a];
    if (!(cs > 0.0)) continue;
    const int hit = ray_elem(w, e, x, om, &t);
    if (!hit) {
      if (!(t > -w->tau && t <= 0.0)) continue;
      t = 0.0;
    }
    if (t <= tmax && (t < best || (t == best && e < be))) {
      best = t;
      be = e;
    }
  }
  *t_out = best;
  return be;
}

typedef struct {
  const wost_t* w;
  const double *g, *hv, *hp, *f;
  double eps;
  int max_steps;
  uint64_t seed;
  uint32_t tag;
  double sqs; /* sqrt(sigma) of the screened equation; 0 = Poisson */
} wost_ctx_t;

/* The Neumann term of one star step (see above). */
static double wost_neumann_term(const wost_ctx_t* c, const double* x, int on_n, int64_t self, double R, uint64_t wid,
                                uint32_t step) {
  const wost_t* w = c->w;
  const int dim = w->dim;
  double total = 0.0;
  for (int64_t q = 0; q < w->n_neu; ++q) {
    const int64_t e = w->neu_ids[q];
    double cp[3];
    if (prim_closest64(&((const obvh_t*)w->all)->m, e, x, cp) < R * R) total += w->meas[e];
  }
  if (!(total > 0.0)) return 0.0;
  double u[4];
  draw(c->seed, wid, step, c->tag + 8u, u);
  const double target = u[0] * total;
  double run = 0.0;
  int64_t pick = -1;
  for (int64_t q = 0; q < w->n_neu; ++q) {
    const int64_t e = w->neu_ids[q];
    double cp[3];
    if (prim_closest64(&((const obvh_t*)w->all)->m, e, x, cp) < R * R) {
      run += w->meas[e];
      pick = e;
      if (run > target) break;
    }
  }
  /* a uniform point on the element */
  const int32_t* f = w->F + pick * dim;
  double z[3] = {0, 0, 0};
  if (dim == 2) {
    for (int a = 0; a < 2; ++a) z[a] = w->V[2 * f[0] + a] + u[1] * (w->V[2 * f[1] + a] - w->V[2 * f[0] + a]);
  } else {
    const double sq = sqrt(u[1]), b1 = sq * (1.0 - u[2]), b2 = sq * u[2];
    for (int a = 0; a < 3; ++a) {
      const double v0 = w->V[3 * f[0] + a];
      z[a] = v0 + b1 * (w->V[3 * f[1] + a] - v0) + b2 * (w->V[3 * f[2] + a] - v0);
    }
  }
  /* the element under an on-boundary x is covered by wost_own_term */
  if (on_n && pick == self) return 0.0;
  double r2 = 0.0, dir[3] = {0, 0, 0};
  for (int a = 0; a < dim; ++a) {
    dir[a] = z[a] - x[a];
    r2 += dir[a] * dir[a];
  }
  const double r = sqrt(r2);
  if (!(r < R) || !(r > 0.0)) return 0.0;
  for (int a = 0; a < dim; ++a) dir[a] /= r;
  /* seen from x: no Neumann crossing strictly before z (z's own element and */
  /* the element under x excluded)                                           */
  for (int64_t q = 0; q < w->n_neu; ++q) {
    const int64_t e = w->neu_ids[q];
    if (e == pick || (on_n && e == self)) continue;
    double th, cs = 0.0;
    for (int a = 0; a < dim; ++a) cs += w->nrm[e * dim + a] * dir[a];
    if (fabs(cs) < 1e-4) continue; /* grazing elements do not occlude */
    if (ray_elem(w, e, x, dir, &th) && th < r * (1.0 - 1e-9)) return 0.0;
  }
  const double gb = orc_ball_green_sigma(dim, c->sqs, R, r);
  const double inv_a = on_n ? 2.0 : 1.0;
  return inv_a * gb * orc_neumann_eval(c->hv, c->hp, dim, z, w->nrm + pick * dim) * total;
}

/* The Neumann term over the element under an on-boundary x, sampled      */
/* around x inside the element, where G^B is singular (a uniform point     */
/* would give the 3D term infinite variance): 2D a side (u0 < 1/2: towards */
/* b) and rho = u1 rho_max, rho_max = min(R, distance to that end); 3D a   */
/* direction theta = 2 pi u0 in the element's plane (e1 = (b - a)/|b - a|,  */
/* e2 = n x e1) and rho = u1 rho_max, rho_max = min(R, distance to the     */
/* triangle's border along it).  1/pdf = 2 rho_max (2D), 2 pi rho rho_max   */
/* (3D); the term is (1/a) G^B(rho) h(z) / pdf with a = 1/2.  Draws:       */
/* Philox (walk id, step - 1, tag + 12).                                    */
static double wost_own_term(const wost_ctx_t* c, const double* x, int64_t self, double R, uint64_t wid,
                            uint32_t step) {
  const wost_t* w = c->w;
  const int dim = w->dim;
  double u[4];
  draw(c->seed, wid, step, c->tag + 12u, u);
  const int32_t* f = w->F + self * dim;
  const double* n = w->nrm + self * dim;
  double z[3] = {0, 0, 0}, rmax, rho;
  if (dim == 2) {
    const double* a = w->V + 2 * (int64_t)f[0];
    const double* b = w->V + 2 * (int64_t)f[1];
    const double len = sqrt((b[0] - a[0]) * (b[0] - a[0]) + (b[1] - a[1]) * (b[1] - a[1]));
    const double t[2] = {(b[0] - a[0]) / len, (b[1] - a[1]) / len};
    double sx = (x[0] - a[0]) * t[0] + (x[1] - a[1]) * t[1];
    sx = fmin(fmax(sx, 0.0), len);
    const double sgn = u[0] < 0.5 ? 1.0 : -1.0;
    rmax = fmin(R, sgn > 0.0 ? len - sx : sx);
    if (!(rmax > 0.0)) return 0.0;
    rho = u[1] * rmax;
    for (int k = 0; k < 2; ++k) z[k] = x[k] + sgn * rho * t[k];
    return 2.0 * orc_ball_green_sigma(dim, c->sqs, R, rho) * orc_neumann_eval(c->hv, c->hp, dim, z, n) * 2.0 * rmax;
  }
  const double* P[3] = {w->V + 3 * (int64_t)f[0], w->V + 3 * (int64_t)f[1], w->V + 3 * (int64_t)f[2]};
  double e1[3], e2[3], d[3];
  double l1 = 0.0;
  for (int k = 0; k < 3; ++k) {
    e1[k] = P[1][k] - P[0][k];
    l1 += e1[k] * e1[k];
  }
  l1 = sqrt(l1);
  for (int k = 0; k < 3; ++k) e1[k] /= l1;
  e2[0] = n[1] * e1[2] - n[2] * e1[1];
  e2[1] = n[2] * e1[0] - n[0] * e1[2];
  e2[2] = n[0] * e1[1] - n[1] * e1[0];
  const double th = 2.0 * ORC_PI * u[0];
  for (int k = 0; k < 3; ++k) d[k] = cos(th) * e1[k] + sin(th) * e2[k];
  rmax = R;
  for (int j = 0; j < 3; ++j) {
    const double* p = P[j];
    const double* q = P[(j + 1) % 3];
    const double pq[3] = {q[0] - p[0], q[1] - p[1], q[2] - p[2]};
    /* in-plane normal of the edge pointing into the triangle */
    const double m[3] = {n[1] * pq[2] - n[2] * pq[1], n[2] * pq[0] - n[0] * pq[2], n[0] * pq[1] - n[1] * pq[0]};
    const double dm = dot3d(d, m);
    if (dm < 0.0) {
      const double xp[3] = {x[0] - p[0], x[1] - p[1], x[2] - p[2]};
      const double lim = dot3d(xp, m) / -dm;
      if (lim < rmax) rmax = lim;
    }
  }
  if (!(rmax > 0.0)) return 0.0;
  rho = u[1] * rmax;
  for (int k = 0; k < 3; ++k) z[k] = x[k] + rho * d[k];
  return 2.0 * orc_ball_green_sigma(dim, c->sqs, R, rho) * orc_neumann_eval(c->hv, c->hp, dim, z, n) *
         (2.0 * ORC_PI * rho * rmax);
}

static void wost_walk_one(const wost_ctx_t* c, const double* x0, int64_t e0, uint64_t wid, double* U_out,
                          double* grad_out, int32_t* steps_out, int32_t* prim_out) {
  const wost_t* w = c->w;
  const int dim = w->dim;
  const int has_f = !fn_is_zero(c->f), has_h = !fn_is_zero(c->hv) || !fn_is_zero(c->hp);
  double x[3] = {0, 0, 0}, pbar[3] = {0, 0, 0}, nu[3] = {0, 0, 0}, nx[3] = {0, 0, 0};
  for (int a = 0; a < dim; ++a) x[a] = x0[a];
  int on_n = e0 >= 0;
  int64_t self = e0;
  if (on_n)
    for (int a = 0; a < dim; ++a) nx[a] = w->nrm[e0 * dim + a];
  double acc = 0.0, wf0 = 0.0, wg0 = 0.0, R0 = 0.0, cv = 0.0;
  /* screened: the walk's throughput (the product of its steps' factors: the */
  /* gradient ball's C, each star step's W(r)) and the gradient ball's C, Qg */
  const double sk = c->sqs;
  double thr = 1.0, C0 = 1.0, Qg0 = 1.0;
  int k = 0;
  int64_t prim = -1;
  for (;;) {
    const double dD = sqrt(bvh_closest((const obvh_t*)w->dir, x, pbar, &prim));
    ++k;
    if (!(dD <= 4.0 * w->diag)) break; /* escaped through a rounding gap: capped */
    if (k == 1) cv = orc_fn_eval(c->g, dim, pbar);
    if (dD < c->eps || k >= c->max_steps) break;
    double u[4];
    draw(c->seed, wid, (uint32_t)(k - 1), c->tag, u);
    double om[3] = {0, 0, 0}, rho, wu, wg;
    if (k == 1 && !on_n) {
      double cp[3];
      int64_t ea;
      const double dA = sqrt(bvh_closest((const obvh_t*)w->all, x, cp, &ea));
      if (dA >= c->eps) {
        /* the gradient ball: B(x, d_all) holds no boundary */
        const double R = dA;
        orc_sphere_step(dim, R, u[0], u[1], u[2], om, &rho, &wu, &wg);
        if (sk > 0.0) {
          orc_screened_factors(dim, sk * R, &C0, &Qg0);
          thr = C0;
        }
        if (has_f) {
          if (sk > 0.0) orc_screened_step_weights(dim, sk, R, rho, &wu, &wg);
          double y[3] = {0, 0, 0};
          for (int a = 0; a < dim; ++a) y[a] = x[a] + rho * om[a];
          const double fy = orc_fn_eval(c->f, dim, y);
          acc += wu * fy;
          wf0 = wu * fy;
          wg0 = wg * fy;
        }
        R0 = R;
        for (int a = 0; a < dim; ++a) {
          nu[a] = om[a];
          x[a] += R * om[a];
        }
        continue;
      }
    }
    /* star step */
    orc_sphere_step(dim, 1.0, u[0], u[1], u[2], om, &rho, &wu, &wg);
    if (on_n) {
      double s = 0.0;
      for (int a = 0; a < dim; ++a) s += nx[a] * om[a];
      if (s > 0.0)
        for (int a = 0; a < dim; ++a) om[a] = -om[a];
    }
    const double dS = wost_sil_dist(w, x);
    double R = dD < dS ? dD : dS;
    if (R < c->eps) R = c->eps;
    double th;
    const int64_t eh = wost_ray(w, x, om, R, on_n ? self : -1, &th);
    const double r = eh >= 0 ? th : R;
    /* this step's source and Neumann terms carry the throughput into it */
    if (has_f && r > 0.0) { /* a crossing at t = 0 leaves no segment */
      const double rr = r * u[2];
      double y[3] = {0, 0, 0};
      for (int a = 0; a < dim; ++a) y[a] = x[a] + rr * om[a];
      /* -|S| r rr^(d-1) G(rr): the ball's weight at rr scaled by r / R */
      double wsrc = dim == 2 ? -r * rr * log(R / rr) : -r * rr * (1.0 - rr / R);
      if (sk > 0.0) {
        double wb, wgb;
        orc_screened_step_weights(dim, sk, R, rr, &wb, &wgb);
        wsrc = (r / R) * wb;
      }
      acc += thr * wsrc * orc_fn_eval(c->f, dim, y);
    }
    if (has_h) {
      acc += thr * wost_neumann_term(c, x, on_n, self, R, wid, (uint32_t)(k - 1));
      if (on_n) acc += thr * wost_own_term(c, x, self, R, wid, (uint32_t)(k - 1));
    }
    if (sk > 0.0) thr *= orc_star_kernel_sigma(dim, sk, R, r);
    if (eh >= 0) {
      for (int a = 0; a < dim; ++a) {
        x[a] += th * om[a];
        nx[a] = w->nrm[eh * dim + a];
      }
      on_n = 1;
      self = eh;
    } else {
      for (int a = 0; a < dim; ++a) x[a] += R * om[a];
      on_n = 0;
      self = -1;
    }
  }
  const double U = thr * orc_fn_eval(c->g, dim, pbar) + acc;
  *U_out = U;
  /* screened: (U - wf0) / C0 estimates u at the gradient ball's sphere point */
  const double s = !(R0 > 0.0) ? 0.0
                   : sk > 0.0  ? ((double)dim / R0) * Qg0 * ((U - wf0) / C0 - cv) + wg0
                               : ((double)dim / R0) * (U - wf0 - cv) + wg0;
  for (int a = 0; a < dim; ++a) grad_out[a] = s * nu[a];
  *steps_out = k;
  *prim_out = prim >= 0 ? (int32_t)w->dir_ids[prim] : -1;
}

/* W walks from each of n starts (start_elem[i] >= 0: the start lies on that */
/* Neumann element; -1: inside).  Walk j of start i has id                   */
/* id_base + i*W + j; outputs per walk: U, grad[dim], steps, the Dirichlet   */
/* element of the end (whole numbering).                                      */
/* sqs = sqrt(sigma) > 0: the screened equation (Delta - sigma) u = f.      */
void orc_wost_walks_sigma(void* h, const double* g, const double* hv, const double* hp, const double* f,
                          double sqs, const float* starts, const int32_t* start_elem, int64_t n, int32_t W,
                          double eps, int32_t max_steps, uint64_t seed, uint64_t id_base, uint32_t tag, double* U,
                          double* grad, int32_t* steps, int32_t* prim) {
  const wost_t* w = (const wost_t*)h;
  const wost_ctx_t c = {w, g, hv, hp, f, eps, max_steps, seed, tag, sqs};
  const int dim = w->dim;
  const int64_t total = n * (int64_t)W;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t t = 0; t < total; ++t) {
    const int64_t i = t / W;
    double x0[3] = {0, 0, 0};
    for (int a = 0; a < dim; ++a) x0[a] = starts[i * dim + a];
    wost_walk_one(&c, x0, start_elem ? start_elem[i] : -1, id_base + (uint64_t)t, &U[t], &grad[t * dim], &steps[t],
                  &prim[t]);
  }
}

void orc_wost_walks(void* h, const double* g, const double* hv, const double* hp, const double* f,
                    const float* starts, const int32_t* start_elem, int64_t n, int32_t W, double eps,
                    int32_t max_steps, uint64_t seed, uint64_t id_base, uint32_t tag, double* U, double* grad,
                    int32_t* steps, int32_t* prim) {
  orc_wost_walks_sigma(h, g, hv, hp, f, 0.0, starts, start_elem, n, W, eps, max_steps, seed, id_base, tag, U, grad,
                       steps, prim);
}

/* Queries for the tests: distances to the Dirichlet part and to the closest */
/* silhouette, and the first Neumann crossing of rays.                        */
void orc_wost_query(void* h, const double* pts, int64_t n, double* d_dir, double* d_sil) {
  const wost_t* w = (const wost_t*)h;
  const int dim = w->dim;
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t i = 0; i < n; ++i) {
    double cp[3];
    int64_t e;
    d_dir[i] = sqrt(bvh_closest((const obvh_t*)w->dir, pts + i * dim, cp, &e));
    d_sil[i] = wost_sil_dist(w, pts + i * dim);
  }
}

void orc_wost_rays(void* h, const double* org, const double* dir, const int32_t* skip, int64_t n, double tmax,
                   double* t_out, int32_t* e_out) {
  const wost_t* w = (const wost_t*)h;
  const int dim = w->dim;
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t i = 0; i < n; ++i) {
    double t;
    const int64_t e = wost_ray(w, org + i * dim, dir + i * dim, tmax, skip ? skip[i] : -1, &t);
    t_out[i] = t;
    e_out[i] = (int32_t)e;
  }
}
