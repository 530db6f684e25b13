// bvc_walk.cu -- walk on spheres (K2 cache walks, K6 pointwise walks), the
// per-start reduction (K3), and the cache build / pointwise estimate entry
// points.
//
// Walk kernel design.  One thread carries one walk at a time; a persistent
// grid (all SMs, as many blocks as fit) pulls walks from a global counter in
// chunks of 128 per warp, and whenever lanes finish their walks the warp
// refills exactly those lanes (warp-level compaction of finished walks).
// A walk step is one BVH closest-point query (stack in shared memory), then
// the step itself (termination test, one Philox draw, sphere sample and,
// when f is non-zero, one source-term evaluation).  Each lane is always in
// one of three states -- at an internal BVH node, at a leaf, or at the step
// -- and on every iteration the warp runs only the most populated kind of
// work (the step once at least half the working lanes wait for it; a node
// iteration descends up to kNodeReps internal nodes per lane, a leaf
// iteration tests up to 1 (3D) or 2 (2D) leaves), so the lanes of a warp
// execute the same instructions instead of diverging along different tree
// paths, and no lane waits for the slowest query in its warp.
// Per-walk results go to FP32 records; K3 reduces them in FP64 in a fixed
// order, so results do not depend on scheduling.
#include <cuda_fp16.h>

#include <cmath>
#include <mutex>

#include "bvc_device.cuh"
#include "bvc_internal.h"

namespace bvc {

// Resident blocks per SM the walk kernel is compiled for (2D: 56 registers,
// 9 x 4 warps, measured best on GB300; 3D needs more registers).
#ifndef BVC_WALK_MINB
#define BVC_WALK_MINB(D) ((D) == 2 ? 9 : 7)
#endif
#ifndef BVC_WALK_POLICY
#define BVC_WALK_POLICY 0
#endif
// Warm-started closest-point queries (previous closest element first).
#ifndef BVC_WALK_WARM
#define BVC_WALK_WARM 1
#endif
// Internal nodes a lane visits per node iteration of the scheduler (measured
// on GB300, cache + pointwise walks of the sphere / star workloads: 1 295 /
// 34.1 ms, 2 286 / 32.6, 3 282 / 31.9, 4 276 / 31.8, 6 281 / 31.7, 8 282 /
// 31.8, 16 297 / 31.6).
#ifndef BVC_WALK_NODE_REPS
#define BVC_WALK_NODE_REPS 4
#endif
constexpr int kNodeReps = BVC_WALK_NODE_REPS;
// Leaves a lane tests per leaf iteration (measured on GB300 with 4 node
// visits: 2D 1 / 2 -> 31.7 / 30.7 ms for the star's cache and pointwise
// walks; 3D 1 / 2 -> 278 / 284 ms on the sphere).
#ifndef BVC_WALK_LEAF_REPS_2D
#define BVC_WALK_LEAF_REPS_2D 2
#endif
#ifndef BVC_WALK_LEAF_REPS_3D
#define BVC_WALK_LEAF_REPS_3D 1
#endif
constexpr int kLeafReps2 = BVC_WALK_LEAF_REPS_2D, kLeafReps3 = BVC_WALK_LEAF_REPS_3D;
constexpr int kWalkBlock = 128;
constexpr int kStack = kTravStack;
constexpr int64_t kChunk = 128;  // default walks per warp refill

struct WalkParams {
  DevGeometry G;
  DevFunction g, f;
  const float* starts;  // [D][pt_stride]
  const float* nrm;     // [D][pt_stride] or null
  int64_t pt_stride;
  int64_t i0;           // first start of this launch
  int32_t W;
  int64_t total;        // walks in this launch
  uint64_t wid0;        // walk id of walk 0 of this launch
  float eps;
  int32_t max_steps;
  uint64_t seed;
  uint32_t tag;
  float* rec;           // planes of `total` floats
  int32_t* steps;       // optional per-walk debug output
  int32_t* prim;
  unsigned long long* counter;
  // First closest-point query of every start of this launch, shared by its
  // walks (they all begin at the same point), or null: planes of
  // (total / W) floats: d2, p - closest (D), element id bits.
  const float* first;
  // Batches of meshes (kRecEnd walks only): the mesh of every start, and the
  // meshes' roots and shells; null for one mesh (root 0, shell eps).
  const int32_t* sample_mesh;
  const BatchMeshDev* meshes;
  // kRecEnd walks: when non-null the seed is read from this device word.
  const uint64_t* seed_dev;
  // Boundary data from vertex values (device float[n_verts]) instead of g.
  const float* gv;
  // kRecAdj walks: adjoint weights dL/du^ and dL/d(du/dn^) of every start
  // (indexed like the starts) and the accumulated gradients with respect to
  // the vertex values of g and the bump amplitudes of f.
  const double* adj_u;
  const double* adj_q;
  double* grad_gv;
  double* grad_amp;
  // screened Poisson: sqrt(sigma) (> 0 selects the screened kernel variant)
  float sqs;
  // launch shape: walks per warp refill (set by launch_walk)
  int64_t chunk;
  int32_t blocks_per_sm;  // 0 = as many as fit
};

// The first query of each start of a launch, once per start.
template <int D>
__global__ void __launch_bounds__(128) k_first_hits(DevGeometry G, const float* __restrict__ starts,
                                                    int64_t pt_stride, int64_t i0, int64_t c, float* __restrict__ fh,
                                                    const int32_t* __restrict__ sample_mesh,
                                                    const BatchMeshDev* __restrict__ meshes) {
  __shared__ int snode[kStack * 128];
  __shared__ float sdist[kStack * 128];
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < c; r += (int64_t)gridDim.x * blockDim.x) {
    float p[D];
#pragma unroll
    for (int a = 0; a < D; ++a) p[a] = starts[a * pt_stride + i0 + r];
    Hit<D> h;
    TravCount tc{0, 0};
    const int root = sample_mesh ? meshes[sample_mesh[i0 + r]].root : 0;
    bvh_closest<D>(G, p, h, snode + threadIdx.x, sdist + threadIdx.x, 128, tc, root);
    fh[r] = h.d2;
#pragma unroll
    for (int a = 0; a < D; ++a) fh[(1 + a) * c + r] = h.df[a];
    fh[(1 + D) * c + r] = __int_as_float(h.id);
  }
}

// Lane states of the walk kernel.
constexpr int kIdle = 0;   // holds no walk
constexpr int kQuery = 1;  // inside a closest-point query (cur = node >= 0 or leaf < 0)
constexpr int kStep = 2;   // query done: termination test, sphere sample, source term

// Record kinds: per walk t, with `total` walks in the launch,
//   kRecGn   rec[t] = U, rec[total + t] = n . grad            (cache walks)
//   kRecGrad rec[t] = U, rec[(1 + a) total + t] = grad_a      (pointwise walks)
//   kRecEnd  rec[a total + t] = closest point at the end (a < D),
//            rec[D total + t] = (D / R0)(n . w0) (0 if the walk stopped at
//            its start); for f = 0 a walk's path does not depend on g, and
//            U = g(end), n . grad = rec[D] (g(end) - g(closest point of start)).
//            With a one-term bump source f = sum_b A_b psi_b (kMaxBumps
//            bumps), also rec[(D + 1 + b) total + t] = sum over steps of
//            w_u psi_b(y) and rec[(D + 1 + kMaxBumps + b) total + t] = bump
//            b's part of the n . grad sample, so that U and n . grad stay
//            linear in (g, A): U = g(end) + sum_b A_b rec[D + 1 + b], etc.
//   kRecAdj  the adjoint replay of a kRecGn walk (same path, same draws):
//            with cu = dL/du^ / W and cq = dL/d(du/dn^) / W of its start,
//            U and n . grad are linear in the vertex values of g and the
//            bump amplitudes A of f, so the walk adds
//              (cu + cq (D/R0)(n . w0)) x (interpolation weights at the end)
//            to dL/dg_vertex, the source terms' derivatives to dL/dA, and
//            writes rec[t] = -cq (D/R0)(n . w0), the weight of the control
//            variate g(closest point of the start), reduced per start later.
constexpr int kRecGn = 0, kRecGrad = 1, kRecEnd = 2, kRecAdj = 3;

// FM: 0 Laplace (f = 0), 1 Poisson with a source term, 2 screened Poisson
// (sigma > 0, f = 0): every ball multiplies the walk's throughput by its
// screened mean-value factor C (value) and the first ball's Qg scales the
// gradient estimate (screened_factors); 3 screened Poisson with a source
// term, each ball's source sample weighted by the screened ball Green's
// function (screened_step_weights) and by the throughput into the ball.
template <int D, int FM, int REC, bool CNT>
__global__ void __launch_bounds__(kWalkBlock, REC == kRecAdj || (REC == kRecEnd && FM == 1) ? 4 : BVC_WALK_MINB(D))
    k_walk(const WalkParams P) {
  constexpr bool HAS_F = FM == 1 || FM == 3;
  constexpr bool SCR = FM >= 2;
  // Traversal stacks: node links and box distances, the latter in FP16
  // rounded down (a smaller stored distance can only cost an extra visit,
  // never prune a box that must be visited).
  __shared__ int snode[kStack * kWalkBlock];
  __shared__ __half sdist[kStack * kWalkBlock];
  int* const stk_node = snode + threadIdx.x;  // entry e at [e * kWalkBlock]
  __half* const stk_dist = sdist + threadIdx.x;
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const float kInf = __int_as_float(0x7f800000);
  const DevGeometry& G = P.G;
  // warp-uniform work queue
  int64_t q_next = 0, q_end = 0;
  bool more = true;
  // walk state
  int phase = kIdle;
  int64_t t = 0, i = 0;
  float x[D], nu[D];
#pragma unroll
  for (int a = 0; a < D; ++a) x[a] = nu[a] = 0.0f;
  float R0 = 0.0f, usrc = 0.0f, wf0 = 0.0f, wg0 = 0.0f, cv = 0.0f;
  int k = 0;
  // the walk's tree and shell (per mesh in a batch)
  int root = 0;
  float eps = P.eps;
  // screened: throughput and the first ball's factors
  float wthr = 1.0f, C0 = 1.0f, Qg0 = 1.0f;
  // adjoint replay: the start's weights, n . w0, FP64 amplitude gradients
  float cu = 0.0f, cq = 0.0f, nw0 = 0.0f;
  double gA[REC == kRecAdj && HAS_F ? kMaxBumps : 1];
#pragma unroll
  for (int b = 0; b < (REC == kRecAdj && HAS_F ? kMaxBumps : 1); ++b) gA[b] = 0.0;
  // end-point walks with a source: per bump b, sum_steps w_u psi_b(y) and
  // the first step's part of the du/dn sample, (n.w0)(w_g - (D/R0) w_u) psi_b
  constexpr int NB = REC == kRecEnd && HAS_F ? kMaxBumps : 1;
  float sbu[NB], sbc[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) sbu[b] = sbc[b] = 0.0f;
  // query state
  int cur = 0, sp = 0;
  float thr = kInf;
  Hit<D> h;
  h.d2 = kInf;
  h.id = 0x7fffffff;
#pragma unroll
  for (int a = 0; a < D; ++a) h.df[a] = 0.0f;
  unsigned long long my_steps = 0, my_capped = 0, my_nodes = 0, my_prims = 0;

  // A new query starts at the root; when the walk's previous closest element
  // is known it is tested first at the new position, so the traversal
  // starts with its distance as the pruning bound (the answer -- the
  // smallest distance, ties to the lowest id -- does not depend on it).
  auto begin_query = [&]() {
    const int32_t qp = h.q;
    phase = kQuery;
    cur = root;
    sp = 0;
    thr = kInf;
    h.d2 = kInf;
    h.id = 0x7fffffff;
    h.q = -1;
    if (BVC_WALK_WARM && qp >= 0) {
      float d2;
      if (D == 2) {
        const float4 S = __ldg(&G.prims[2 * qp]), T = __ldg(&G.prims[2 * qp + 1]);
        d2 = seg_d2(S, T.x, x[0], x[D - 1]);
        h.id = __float_as_int(T.y);
      } else {
        const float4 A = __ldg(&G.prims[3 * qp]), B = __ldg(&G.prims[3 * qp + 1]), Cq = __ldg(&G.prims[3 * qp + 2]);
        float df[3];
        d2 = tri_closest(A, B, Cq, x, df);
#pragma unroll
        for (int a = 0; a < D; ++a) h.df[a] = df[D == 3 ? a : 0];
        h.id = __float_as_int(A.w);
      }
      h.d2 = d2;
      h.q = qp;
      const float sr = sqrtf(d2) + G.tau;
      thr = sr * sr;
    }
  };
  // Next stacked item still within reach, else the query is complete.
  auto pop = [&]() {
    while (sp > 0) {
      --sp;
      if (__half2float(stk_dist[sp * kWalkBlock]) <= thr) {
        cur = stk_node[sp * kWalkBlock];
        return;
      }
    }
    phase = kStep;
  };

  for (;;) {
    // ---- refill lanes without a walk (warp-converged)
    unsigned need = __ballot_sync(FULL, phase == kIdle);
    while (need != 0u && more) {
      if (q_next >= q_end) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(P.counter, (unsigned long long)P.chunk);
        base = __shfl_sync(FULL, base, 0);
        if ((int64_t)base >= P.total) {
          more = false;
          break;
        }
        q_next = (int64_t)base;
        q_end = min64((int64_t)base + P.chunk, P.total);
      }
      const int avail = (int)min64(q_end - q_next, (int64_t)__popc(need));
      const int rank = __popc(need & ((1u << lane) - 1u));
      if (phase == kIdle && rank < avail) {
        t = q_next + rank;
        const int64_t r = t / P.W;
        i = P.i0 + r;
#pragma unroll
        for (int a = 0; a < D; ++a) x[a] = P.starts[a * P.pt_stride + i];
        if (REC == kRecEnd && P.sample_mesh != nullptr) {
          const BatchMeshDev* M = P.meshes + P.sample_mesh[i];
          root = M->root;
          eps = M->eps;
        }
        if (REC == kRecAdj) {
          cu = (float)(P.adj_u[i] / (double)P.W);
          cq = (float)(P.adj_q[i] / (double)P.W);
        }
        k = 0;
        R0 = usrc = wf0 = wg0 = cv = 0.0f;
        if (SCR) wthr = C0 = Qg0 = 1.0f;
        if (REC == kRecEnd && HAS_F)
#pragma unroll
          for (int b = 0; b < NB; ++b) sbu[b] = sbc[b] = 0.0f;
        if (P.first) {
          const int64_t c = P.total / P.W;
          h.d2 = P.first[r];
#pragma unroll
          for (int a = 0; a < D; ++a) h.df[a] = P.first[(1 + a) * c + r];
          h.id = __float_as_int(P.first[(1 + D) * c + r]);
          h.q = -1;  // closest-point vector already final
          phase = kStep;
        } else {
          h.q = -1;  // no previous element for a new walk
          begin_query();
        }
      }
      q_next += avail;
      need = __ballot_sync(FULL, phase == kIdle);
    }
    // ---- pick the most populated kind of work; the whole warp runs only it
    const unsigned m_node = __ballot_sync(FULL, phase == kQuery && cur >= 0);
    const unsigned m_leaf = __ballot_sync(FULL, phase == kQuery && cur < 0);
    const unsigned m_step = __ballot_sync(FULL, phase == kStep);
    const int nn = __popc(m_node), nl = __popc(m_leaf), ns = __popc(m_step);
    if (nn + nl + ns == 0) break;
    int choice;
    bool take_step;
    if (BVC_WALK_POLICY == 1)
      take_step = ns >= nn && ns >= nl;
    else if (BVC_WALK_POLICY == 2)
      take_step = 3 * ns >= nn + nl + ns;
    else
      take_step = 2 * ns >= nn + nl + ns;
    if (ns > 0 && (take_step || nn + nl == 0))
      choice = kStep;
    else
      choice = nl > nn ? 1 : 0;

    if (choice == 0) {
      // ---- up to kNodeReps internal nodes: order the children, descend into the nearer
#pragma unroll 1
      for (int rep = 0; rep < kNodeReps; ++rep) {
        if (!(phase == kQuery && cur >= 0)) break;
        if (CNT) ++my_nodes;
        int32_t cl, cr;
        float dl, dr;
        node_bounds<D>(G, cur, x, dl, dr, cl, cr);
        if (dr < dl) {
          const int32_t tc = cl;
          cl = cr;
          cr = tc;
          const float td = dl;
          dl = dr;
          dr = td;
        }
        const bool tl = dl <= thr, tr = dr <= thr;
        if (tl && tr) {
          if (!dbg_bad(G, sp >= kStack)) {
            stk_node[sp * kWalkBlock] = cr;
            stk_dist[sp * kWalkBlock] = __float2half_rd(dr);
            ++sp;
          }
          cur = cl;
        } else if (tl) {
          cur = cl;
        } else if (tr) {
          cur = cr;
        } else {
          pop();
        }
      }
    } else if (choice == 1) {
      // ---- up to kLeafReps leaves: canonical FP32 distances, ties to the lowest index
#pragma unroll 1
      for (int rep = 0; rep < (D == 2 ? kLeafReps2 : kLeafReps3); ++rep) {
        if (!(phase == kQuery && cur < 0)) break;
        TravCount tc{0, 0};
        test_leaf<D, CNT>(G, cur, x, h, thr, tc);
        if (CNT) my_prims += tc.prims;
        pop();
      }
    } else {
      // ---- walk step on the finished query
      if (phase == kStep) {
        ++k;
        finish_hit<D>(G, x, h);
        float pbar[D];
#pragma unroll
        for (int a = 0; a < D; ++a) pbar[a] = x[a] - h.df[a];
        const float d = sqrtf(h.d2);
        if ((REC == kRecGn || REC == kRecGrad) && k == 1)
          cv = P.gv ? vertex_g<D>(G, P.gv, h.id, pbar) : eval_fn<D, true>(P.g, pbar);
        if (d < eps || k >= P.max_steps) {
          if (REC == kRecEnd) {
#pragma unroll
            for (int a = 0; a < D; ++a) P.rec[a * P.total + t] = pbar[a];
            float nn2 = 0.0f;
#pragma unroll
            for (int a = 0; a < D; ++a) nn2 = fmaf(P.nrm[a * P.pt_stride + i], nu[a], nn2);
            const float sj = k > 1 ? ((float)D / R0) * nn2 : 0.0f;
            P.rec[D * P.total + t] = sj;
            if (HAS_F)
#pragma unroll
              for (int b = 0; b < NB; ++b) {
                P.rec[(D + 1 + b) * P.total + t] = sbu[b];
                P.rec[(D + 1 + kMaxBumps + b) * P.total + t] = k > 1 ? fmaf(sj, sbu[b], sbc[b]) : 0.0f;
              }
          } else if (REC == kRecAdj) {
            const float s0 = k > 1 ? cq * ((float)D / R0) * nw0 : 0.0f;
            int32_t vid[D];
            float wv[D];
            vertex_weights<D>(G, h.id, pbar, vid, wv);
#pragma unroll
            for (int a = 0; a < D; ++a) atomicAdd(&P.grad_gv[vid[a]], (double)((cu + s0) * wv[a]));
            P.rec[t] = -s0;
          } else {
            const float gend = P.gv ? vertex_g<D>(G, P.gv, h.id, pbar) : eval_fn<D, true>(P.g, pbar);
            const float U = (k == 1 ? cv : (SCR ? wthr * gend : gend)) + usrc;
            // screened: (U - wf0) / C0 estimates u at the first sphere point
            const float sc = k > 1 ? (SCR ? fmaf(((float)D / R0) * Qg0, (U - wf0) / C0 - cv, wg0)
                                          : ((float)D / R0) * (U - wf0 - cv) + wg0)
                                   : 0.0f;
            P.rec[t] = U;
            if (REC == kRecGn) {
              float nn2 = 0.0f;
#pragma unroll
              for (int a = 0; a < D; ++a) nn2 = fmaf(P.nrm[a * P.pt_stride + i], nu[a], nn2);
              P.rec[P.total + t] = sc * nn2;
            } else {
#pragma unroll
              for (int a = 0; a < D; ++a) P.rec[(1 + a) * P.total + t] = sc * nu[a];
            }
          }
          if (P.steps) P.steps[t] = k;
          if (P.prim) P.prim[t] = h.id;
          my_steps += (unsigned long long)k;
          if (!(d < eps)) ++my_capped;
          phase = kIdle;
        } else {
          const float R = d;
          const float thr_in = wthr;  // screened: the throughput into this ball weighs its source term
          if (SCR) {
            float Cs, Qs;
            screened_factors<D>(P.sqs * R, Cs, Qs);
            wthr *= Cs;
            if (k == 1) {
              C0 = Cs;
              Qg0 = Qs;
            }
          }
          const uint64_t seed = (REC == kRecEnd && P.seed_dev != nullptr) ? __ldg(P.seed_dev) : P.seed;
          const U4 r = philox_draw(seed, P.wid0 + (uint64_t)t, (uint32_t)(k - 1), P.tag);
          const float u0 = u01f(r.x);
          float om[D];
          if (D == 2) {
            float sn, cs;
            sincospif(2.0f * u0, &sn, &cs);
            om[0] = cs;
            om[D - 1] = sn;
          } else {
            const float u1 = u01f(r.y);
            const float zc = 1.0f - 2.0f * u0;
            const float st = 2.0f * sqrtf(u0 * (1.0f - u0));
            float sn, cs;
            sincospif(2.0f * u1, &sn, &cs);
            om[0] = st * cs;
            om[1] = st * sn;
            om[D - 1] = zc;
          }
          if (REC == kRecAdj && k == 1) {
            float nn2 = 0.0f;
#pragma unroll
            for (int a = 0; a < D; ++a) nn2 = fmaf(P.nrm[a * P.pt_stride + i], om[a], nn2);
            nw0 = nn2;
          }
          if (HAS_F && REC == kRecEnd) {
            // the source terms per bump (Sec. 3.1 ball Green's function
            // weights, as the single right-hand side walk draws them)
            const float u2 = u01f(r.z);
            const float rho = R * u2;
            float y[D];
#pragma unroll
            for (int a = 0; a < D; ++a) y[a] = fmaf(rho, om[a], x[a]);
            const float wu = D == 2 ? R * rho * __logf(u2) : -rho * (R - rho);
            float psi[kMaxBumps];
            bump_shapes<D>(P.f, y, psi);
#pragma unroll
            for (int b = 0; b < NB; ++b) sbu[b] = fmaf(wu, psi[b], sbu[b]);
            if (k == 1) {
              float nn2 = 0.0f;
#pragma unroll
              for (int a = 0; a < D; ++a) nn2 = fmaf(P.nrm[a * P.pt_stride + i], om[a], nn2);
              const float q = D == 2 ? u2 * u2 : u2 * u2 * u2;
              const float c1 = nn2 * fmaf(-((float)D / R), wu, -R * (1.0f - q));
#pragma unroll
              for (int b = 0; b < NB; ++b) sbc[b] = c1 * psi[b];
            }
          } else if (HAS_F && REC == kRecAdj) {
            // d/dA_k of the source terms: U gains w_u psi_k(y) at every step;
            // n.grad gains (D/R0)(n.w0) w_u psi_k(y) at steps after the first
            // and (n.w0) w_g psi_k(y0) at the first (w_g = -R (1 - (rho/R)^D))
            const float u2 = u01f(r.z);
            const float rho = R * u2;
            float y[D];
#pragma unroll
            for (int a = 0; a < D; ++a) y[a] = fmaf(rho, om[a], x[a]);
            const float wu = D == 2 ? R * rho * __logf(u2) : -rho * (R - rho);
            float coef;
            if (k == 1) {
              const float q = D == 2 ? u2 * u2 : u2 * u2 * u2;
              coef = fmaf(cq * nw0, -R * (1.0f - q), cu * wu);
            } else {
              coef = fmaf(cq * nw0, (float)D / R0, cu) * wu;
            }
            float psi[kMaxBumps];
            bump_shapes<D>(P.f, y, psi);
#pragma unroll
            for (int b = 0; b < (REC == kRecAdj && HAS_F ? kMaxBumps : 1); ++b) gA[b] += (double)(coef * psi[b]);
          } else if (HAS_F) {
            const float u2 = u01f(r.z);
            const float rho = R * u2;
            float y[D];
#pragma unroll
            for (int a = 0; a < D; ++a) y[a] = fmaf(rho, om[a], x[a]);
            const float fy = eval_fn<D, true>(P.f, y);
            // ball Green's function weights: -R rho ln(R/rho) (2D), -rho (R - rho) (3D)
            float wu = D == 2 ? R * rho * __logf(u2) : -rho * (R - rho), wg = 0.0f;
            if (SCR) screened_step_weights<D>(P.sqs, R, rho, k == 1, wu, wg);
            usrc = fmaf(SCR ? thr_in * wu : wu, fy, usrc);
            if (k == 1) {
              wf0 = wu * fy;
              const float q = D == 2 ? u2 * u2 : u2 * u2 * u2;
              wg0 = (SCR ? wg : -R * (1.0f - q)) * fy;
            }
          }
          if (k == 1) {
            R0 = R;
#pragma unroll
            for (int a = 0; a < D; ++a) nu[a] = om[a];
          }
#pragma unroll
          for (int a = 0; a < D; ++a) x[a] = fmaf(R, om[a], x[a]);
          begin_query();
        }
      }
    }
  }
  // one atomic per warp for the step and cap counters
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    my_steps += __shfl_xor_sync(FULL, my_steps, o);
    my_capped += __shfl_xor_sync(FULL, my_capped, o);
    if (CNT) {
      my_nodes += __shfl_xor_sync(FULL, my_nodes, o);
      my_prims += __shfl_xor_sync(FULL, my_prims, o);
    }
  }
  if (REC == kRecAdj && HAS_F) {
#pragma unroll
    for (int b = 0; b < (REC == kRecAdj && HAS_F ? kMaxBumps : 1); ++b) {
      double v = gA[b];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
      if (lane == 0 && v != 0.0) atomicAdd(&P.grad_amp[b], v);
    }
  }
  if (lane == 0) {
    if (my_steps) atomicAdd(&P.G.stats[kStatSteps], my_steps);
    if (my_capped) atomicAdd(&P.G.stats[kStatCapped], my_capped);
    if (CNT) {
      atomicAdd(&P.G.stats[kStatNodes], my_nodes);
      atomicAdd(&P.G.stats[kStatPrims], my_prims);
    }
  }
}

// K3: one warp per start; lanes stride the start's walks, FP64 partials are
// combined by a fixed xor-shuffle tree (deterministic).
__global__ void __launch_bounds__(256) k_reduce(const ReduceParams R) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < R.n; i += nwarps) {
    for (int p = 0; p < R.planes; ++p) {
      const float* r = R.rec + p * R.stride + i * R.W;
      double s = 0.0;
      for (int j = lane; j < R.W; j += 32) s += (double)r[j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) {
        if (R.mode == 0)
          R.out[p][i] = s / (double)R.W;
        else
          R.out[p][i] += s;
      }
    }
  }
}

template <int D, int FM, int REC>
static const void* walk_kernel(bool cnt) {
  return cnt ? (const void*)k_walk<D, FM, REC, true> : (const void*)k_walk<D, FM, REC, false>;
}

// rec: kRecGn / kRecGrad / kRecEnd (f = 0, or a one-term bump source with
// per-bump records) / kRecAdj (no counting); scr: screened Poisson (kRecGn /
// kRecGrad, with or without a source).
static const void* pick_walk(int dim, bool has_f, int rec, bool cnt, bool scr = false) {
  if (rec == kRecEnd) {
    if (has_f) return dim == 2 ? walk_kernel<2, 1, kRecEnd>(cnt) : walk_kernel<3, 1, kRecEnd>(cnt);
    return dim == 2 ? walk_kernel<2, 0, kRecEnd>(cnt) : walk_kernel<3, 0, kRecEnd>(cnt);
  }
  if (rec == kRecAdj) {
    if (dim == 2) return has_f ? (const void*)k_walk<2, 1, kRecAdj, false> : (const void*)k_walk<2, 0, kRecAdj, false>;
    return has_f ? (const void*)k_walk<3, 1, kRecAdj, false> : (const void*)k_walk<3, 0, kRecAdj, false>;
  }
  const bool gn = rec == kRecGn;
  if (scr) {
    if (has_f) {
      if (dim == 2) return gn ? walk_kernel<2, 3, kRecGn>(cnt) : walk_kernel<2, 3, kRecGrad>(cnt);
      return gn ? walk_kernel<3, 3, kRecGn>(cnt) : walk_kernel<3, 3, kRecGrad>(cnt);
    }
    if (dim == 2) return gn ? walk_kernel<2, 2, kRecGn>(cnt) : walk_kernel<2, 2, kRecGrad>(cnt);
    return gn ? walk_kernel<3, 2, kRecGn>(cnt) : walk_kernel<3, 2, kRecGrad>(cnt);
  }
  if (dim == 2) {
    if (has_f) return gn ? walk_kernel<2, 1, kRecGn>(cnt) : walk_kernel<2, 1, kRecGrad>(cnt);
    return gn ? walk_kernel<2, 0, kRecGn>(cnt) : walk_kernel<2, 0, kRecGrad>(cnt);
  }
  if (has_f) return gn ? walk_kernel<3, 1, kRecGn>(cnt) : walk_kernel<3, 1, kRecGrad>(cnt);
  return gn ? walk_kernel<3, 0, kRecGn>(cnt) : walk_kernel<3, 0, kRecGrad>(cnt);
}

static bvc_status launch_walk(int dim, bool has_f, int rec, bool cnt, const WalkParams& P0, cudaStream_t s) {
  WalkParams P = P0;
  if (P.chunk < 1) P.chunk = kChunk;
  const void* kern = pick_walk(dim, has_f, rec, cnt, P.sqs > 0.0f);
  const int64_t want = (P.total + 31) / 32;
  int bps = max_blocks_per_sm(kern, kWalkBlock, 0);
  if (P.blocks_per_sm > 0 && P.blocks_per_sm < bps) bps = P.blocks_per_sm;
  int grid = num_sms() * bps;
  const int64_t need_blocks = (want + kWalkBlock / 32 - 1) / (kWalkBlock / 32);
  if (need_blocks < grid) grid = (int)(need_blocks > 0 ? need_blocks : 1);
  BVC_CUDA_TRY(cudaMemsetAsync(P.counter, 0, sizeof(unsigned long long), s));
  void* args[] = {(void*)&P};
  ProfScope ps("walk", s);
  BVC_CUDA_TRY(cudaLaunchKernel(kern, dim3(grid), dim3(kWalkBlock), args, 0, s));
  return BVC_OK;
}

static bvc_status launch_first_hits(int dim, const DevGeometry& G, const float* starts, int64_t pt_stride, int64_t i0,
                                    int64_t c, float* fh, cudaStream_t s, const int32_t* sample_mesh = nullptr,
                                    const BatchMeshDev* meshes = nullptr) {
  int64_t blocks = (c + 127) / 128;
  const int64_t cap = (int64_t)num_sms() * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  ProfScope ps("first_hits", s);
  if (dim == 2)
    k_first_hits<2><<<(unsigned)blocks, 128, 0, s>>>(G, starts, pt_stride, i0, c, fh, sample_mesh, meshes);
  else
    k_first_hits<3><<<(unsigned)blocks, 128, 0, s>>>(G, starts, pt_stride, i0, c, fh, sample_mesh, meshes);
  BVC_LAUNCH_CHECK();
  return BVC_OK;
}

bvc_status launch_reduce(const ReduceParams& R, cudaStream_t s) {
  const int64_t warps = R.n;
  int64_t blocks = (warps * 32 + 255) / 256;
  const int64_t cap = (int64_t)num_sms() * 16;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  ProfScope ps("reduce_walks", s);
  k_reduce<<<(int)blocks, 256, 0, s>>>(R);
  BVC_LAUNCH_CHECK();
  return BVC_OK;
}

// Source candidates of a cache build: G0 x G1 (2D) or G0 x G1 x G2 (3D).
static int64_t src_candidates(const bvc_cache_opts* o, int dim) {
  return (int64_t)o->src_grid[0] * o->src_grid[1] * (dim == 3 ? o->src_grid[2] : 1);
}

static bool valid_walk_args(float eps, int32_t max_steps, int32_t walks) {
  return std::isfinite(eps) && eps > 0.0f && max_steps >= 1 && walks >= 1;
}

}  // namespace bvc

using namespace bvc;

static bvc_status bvc_walk_impl(bvc_geometry g, const bvc_function* gfn, const bvc_function* ffn, const float* starts,
                               const float* nrm, int64_t n, int32_t walks, float eps, int32_t max_steps,
                               uint64_t seed, uint64_t id_base, uint32_t tag, float* rec, int32_t* steps,
                               int32_t* prim, bvc_stream stream) {
  if (g == nullptr || n < 0 || !valid_walk_args(eps, max_steps, walks)) return BVC_ERR_INVALID_ARG;
  if (n == 0) return BVC_OK;
  if (starts == nullptr || rec == nullptr) return BVC_ERR_INVALID_ARG;
  WalkParams P{};
  P.G = g->dev;
  P.chunk = g->tune_chunk;
  P.blocks_per_sm = g->tune_blocks_per_sm;
  if (!make_dev_function(gfn, g->dim, &P.g) || !make_dev_function(ffn, g->dim, &P.f)) return BVC_ERR_INVALID_ARG;
  P.starts = starts;
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
  // the work counter lives in the status block's spare word
  P.counter = g->dev.stats + 3;
  return launch_walk(g->dim, P.f.n_terms > 0, nrm != nullptr ? kRecGn : kRecGrad, g->counting != 0, P,
                     (cudaStream_t)stream);
}
extern "C" bvc_status bvc_walk(bvc_geometry g, const bvc_function* gfn, const bvc_function* ffn, const float* starts,
                               const float* nrm, int64_t n, int32_t walks, float eps, int32_t max_steps,
                               uint64_t seed, uint64_t id_base, uint32_t tag, float* rec, int32_t* steps,
                               int32_t* prim, bvc_stream stream) {
  return bvc::note_status(bvc_walk_impl(g, gfn, ffn, starts, nrm, n, walks, eps, max_steps, seed, id_base, tag, rec, steps, prim, stream));
}

static bvc_status bvc_reduce_walks_impl(const float* rec, int64_t n, int32_t walks, int32_t planes, int32_t mode,
                                       double* out, bvc_stream stream) {
  if (rec == nullptr || out == nullptr || n < 0 || walks < 1 || planes < 0 || planes > 3 || (mode != 0 && mode != 1))
    return BVC_ERR_INVALID_ARG;
  if (n == 0) return BVC_OK;
  ReduceParams R{};
  R.rec = rec;
  R.n = n;
  R.W = walks;
  R.planes = 1 + planes;
  R.stride = n * (int64_t)walks;
  R.mode = mode;
  for (int p = 0; p < R.planes; ++p) R.out[p] = out + p * n;
  return launch_reduce(R, (cudaStream_t)stream);
}
extern "C" bvc_status bvc_reduce_walks(const float* rec, int64_t n, int32_t walks, int32_t planes, int32_t mode,
                                       double* out, bvc_stream stream) {
  return bvc::note_status(bvc_reduce_walks_impl(rec, n, walks, planes, mode, out, stream));
}

// Workspace layout for the chunked drivers: [0, 256) work counter, then the
// first hits of the chunk's starts, then (256-byte aligned) the walk records.
static constexpr size_t kWsHead = 256;
static size_t ws_per_start(int dim, int32_t walks, int planes) {
  return (size_t)walks * (1 + planes) * sizeof(float) + (size_t)(2 + dim) * sizeof(float);
}
static int64_t ws_chunk(size_t ws_bytes, size_t per_start) {
  return ws_bytes < 2 * kWsHead + per_start ? 0 : (int64_t)((ws_bytes - 2 * kWsHead) / per_start);
}
static float* ws_first(void* ws) { return (float*)((char*)ws + kWsHead); }
static float* ws_records(void* ws, int64_t c, int dim) {
  const size_t off = kWsHead + (((size_t)c * (2 + dim) * sizeof(float) + kWsHead - 1) / kWsHead) * kWsHead;
  return (float*)((char*)ws + off);
}

static bvc_status bvc_cache_build_workspace_size_impl(bvc_geometry g, const bvc_cache_opts* opts, size_t* min_bytes,
                                                     size_t* full_bytes) {
  if (g == nullptr || opts == nullptr || opts->n_samples < 0 || opts->walks_per_sample < 1)
    return BVC_ERR_INVALID_ARG;
  const size_t per_sample = ws_per_start(g->dim, opts->walks_per_sample, 1);
  size_t src = 0;
  const int64_t ncand = src_candidates(opts, g->dim);
  if (ncand > 0) bvc_sample_source_workspace_size(ncand, &src);
  const size_t mn = 2 * kWsHead + per_sample, full = 2 * kWsHead + per_sample * (size_t)opts->n_samples;
  if (min_bytes) *min_bytes = mn > src ? mn : src;
  if (full_bytes) *full_bytes = full > src ? full : src;
  return BVC_OK;
}
extern "C" bvc_status bvc_cache_build_workspace_size(bvc_geometry g, const bvc_cache_opts* opts, size_t* min_bytes,
                                                     size_t* full_bytes) {
  return bvc::note_status(bvc_cache_build_workspace_size_impl(g, opts, min_bytes, full_bytes));
}

// g: the domain's geometry (walks); gs: the geometry the samples lie on and
// the source samples fill -- g itself, or a region of interest inside the
// domain (Sec. 3.2 "Boundary Specification"), whose samples may sit on its
// boundary (offset 0).
static bvc_status cache_build(bvc_geometry g, bvc_geometry gs, const bvc_function* gfn, const float* gv,
                              const bvc_function* ffn, const bvc_cache_opts* opts, bvc_cache* cache, void* workspace,
                              size_t workspace_bytes, bvc_stream stream) {
  if (g == nullptr || gs == nullptr || opts == nullptr || cache == nullptr || gs->dim != g->dim)
    return BVC_ERR_INVALID_ARG;
  const int D = g->dim;
  const int64_t N = opts->n_samples;
  const int32_t W = opts->walks_per_sample;
  if (cache->dim != D || cache->n != N || N < 1 || !valid_walk_args((float)opts->eps, opts->max_steps, W) ||
      !(gs == g ? opts->offset_l > 0.0 : opts->offset_l >= 0.0) || cache->z == nullptr || cache->nrm == nullptr ||
      cache->jac == nullptr || cache->u_hat == nullptr ||
      cache->dudn_hat == nullptr || cache->packed == nullptr || workspace == nullptr)
    return BVC_ERR_INVALID_ARG;
  const int64_t ncand = src_candidates(opts, D);
  if (ncand != cache->n_src_cand || ncand < 0) return BVC_ERR_INVALID_ARG;
  if (!std::isfinite(opts->sigma) || opts->sigma < 0.0 || !std::isfinite(opts->clamp_c) || opts->clamp_c < 0.0)
    return BVC_ERR_INVALID_ARG;
  WalkParams P{};
  P.G = g->dev;
  P.chunk = g->tune_chunk;
  P.blocks_per_sm = g->tune_blocks_per_sm;
  P.gv = gv;
  P.sqs = (float)std::sqrt(opts->sigma);
  cache->sigma = opts->sigma;
  cache->clamp_c = opts->clamp_c;
  if (!make_dev_function(gfn, D, &P.g) || !make_dev_function(ffn, D, &P.f)) return BVC_ERR_INVALID_ARG;
  const size_t per_sample = ws_per_start(D, W, 1);
  int64_t chunk = ws_chunk(workspace_bytes, per_sample);
  if (chunk < 1) return BVC_ERR_WORKSPACE;
  if (chunk > N) chunk = N;
  cudaStream_t s = (cudaStream_t)stream;
  cache->bnd_measure = gs->measure;
  bvc_status st =
      bvc_sample_boundary(gs, N, opts->offset_l, opts->seed, cache->z, cache->nrm, cache->jac, nullptr, stream);
  if (st != BVC_OK) return st;
  P.starts = cache->z;
  P.nrm = cache->nrm;
  P.pt_stride = N;
  P.W = W;
  P.eps = (float)opts->eps;
  P.max_steps = opts->max_steps;
  P.seed = opts->seed;
  P.tag = 0;
  P.counter = (unsigned long long*)workspace;
  for (int64_t i0 = 0; i0 < N; i0 += chunk) {
    const int64_t c = (N - i0) < chunk ? (N - i0) : chunk;
    P.i0 = i0;
    P.total = c * (int64_t)W;
    P.wid0 = opts->walk_id_base + (uint64_t)i0 * (uint64_t)W;
    float* fh = ws_first(workspace);
    P.rec = ws_records(workspace, c, D);
    P.first = fh;
    st = launch_first_hits(D, g->dev, P.starts, N, i0, c, fh, s);
    if (st != BVC_OK) return st;
    st = launch_walk(D, P.f.n_terms > 0, kRecGn, g->counting != 0, P, s);
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
    st = opts->reuse_sources ? bvc_source_reweight(gs, ffn, cache, s)
                             : bvc_sample_source(gs, ffn, opts->src_grid, opts->seed, opts->offset_l, cache, workspace,
                                                 workspace_bytes, stream);
    if (st != BVC_OK) return st;
  }
  return bvc_cache_pack(cache, stream);
}

static bvc_status bvc_cache_build_impl(bvc_geometry g, const bvc_function* gfn, const bvc_function* ffn,
                                      const bvc_cache_opts* opts, bvc_cache* cache, void* workspace,
                                      size_t workspace_bytes, bvc_stream stream) {
  return cache_build(g, g, gfn, nullptr, ffn, opts, cache, workspace, workspace_bytes, stream);
}
extern "C" bvc_status bvc_cache_build(bvc_geometry g, const bvc_function* gfn, const bvc_function* ffn,
                                      const bvc_cache_opts* opts, bvc_cache* cache, void* workspace,
                                      size_t workspace_bytes, bvc_stream stream) {
  return bvc::note_status(bvc_cache_build_impl(g, gfn, ffn, opts, cache, workspace, workspace_bytes, stream));
}

static bvc_status bvc_cache_build_region_impl(bvc_geometry domain, bvc_geometry region, const bvc_function* gfn,
                                             const bvc_function* ffn, const bvc_cache_opts* opts, bvc_cache* cache,
                                             void* workspace, size_t workspace_bytes, bvc_stream stream) {
  return cache_build(domain, region, gfn, nullptr, ffn, opts, cache, workspace, workspace_bytes, stream);
}
extern "C" bvc_status bvc_cache_build_region(bvc_geometry domain, bvc_geometry region, const bvc_function* gfn,
                                             const bvc_function* ffn, const bvc_cache_opts* opts, bvc_cache* cache,
                                             void* workspace, size_t workspace_bytes, bvc_stream stream) {
  return bvc::note_status(bvc_cache_build_region_impl(domain, region, gfn, ffn, opts, cache, workspace, workspace_bytes, stream));
}

static bvc_status bvc_cache_build_vg_impl(bvc_geometry g, const float* g_vertex, const bvc_function* ffn,
                                         const bvc_cache_opts* opts, bvc_cache* cache, void* workspace,
                                         size_t workspace_bytes, bvc_stream stream) {
  if (g_vertex == nullptr) return BVC_ERR_INVALID_ARG;
  return cache_build(g, g, nullptr, g_vertex, ffn, opts, cache, workspace, workspace_bytes, stream);
}
extern "C" bvc_status bvc_cache_build_vg(bvc_geometry g, const float* g_vertex, const bvc_function* ffn,
                                         const bvc_cache_opts* opts, bvc_cache* cache, void* workspace,
                                         size_t workspace_bytes, bvc_stream stream) {
  return bvc::note_status(bvc_cache_build_vg_impl(g, g_vertex, ffn, opts, cache, workspace, workspace_bytes, stream));
}

// ---------------------------------------------------------------------------
// Adjoint of the cache build (K2 transposed).  The estimator is linear in
// the vertex values of g and the bump amplitudes of f and the walk paths do
// not depend on either, so the walks are replayed from their Philox streams
// with the adjoint weights of their starts (kRecAdj), and the control
// variate's weights are summed per start and spread over the vertices of the
// element holding the start's first closest point.
__global__ void __launch_bounds__(256) k_adj_cv(const float* __restrict__ rec, int64_t c, int32_t W,
                                               const float* __restrict__ starts, int64_t pt_stride, int64_t i0,
                                               const float* __restrict__ fh, DevGeometry G, int dim,
                                               double* __restrict__ grad_gv) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < c; r += nwarps) {
    double s = 0.0;
    for (int j = lane; j < W; j += 32) s += (double)rec[r * W + j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0 && s != 0.0) {
      const int32_t e = __float_as_int(fh[(1 + dim) * c + r]);
      float p[3];
      for (int a = 0; a < dim; ++a) p[a] = starts[a * pt_stride + i0 + r] - fh[(1 + a) * c + r];
      int32_t vid[3];
      float w[3];
      if (dim == 2)
        vertex_weights<2>(G, e, p, vid, w);
      else
        vertex_weights<3>(G, e, p, vid, w);
      for (int a = 0; a < dim; ++a) atomicAdd(&grad_gv[vid[a]], s * (double)w[a]);
    }
  }
}

// The differentiable source: no term, or one GAUSS / GAUSS_LAPLACIAN term of
// at most kMaxBumps bumps whose amplitudes are the parameters.
static bool diff_source_ok(const bvc_function* ffn, int dim) {
  if (ffn == nullptr || ffn->n_terms == 0) return true;
  if (ffn->n_terms != 1) return false;
  const bvc_term& t = ffn->terms[0];
  if (t.kind != BVC_FN_GAUSS && t.kind != BVC_FN_GAUSS_LAPLACIAN) return false;
  return t.n_coeffs >= 1 && (t.n_coeffs - 1) % (1 + dim) == 0 && (t.n_coeffs - 1) / (1 + dim) <= kMaxBumps;
}

static bvc_status bvc_cache_adjoint_workspace_size_impl(bvc_geometry g, const bvc_cache_opts* opts, size_t* min_bytes,
                                                       size_t* full_bytes) {
  if (g == nullptr || opts == nullptr || opts->n_samples < 1 || opts->walks_per_sample < 1) return BVC_ERR_INVALID_ARG;
  const size_t per = ws_per_start(g->dim, opts->walks_per_sample, 0);
  if (min_bytes) *min_bytes = 2 * kWsHead + per;
  if (full_bytes) *full_bytes = 2 * kWsHead + per * (size_t)opts->n_samples;
  return BVC_OK;
}
extern "C" bvc_status bvc_cache_adjoint_workspace_size(bvc_geometry g, const bvc_cache_opts* opts, size_t* min_bytes,
                                                       size_t* full_bytes) {
  return bvc::note_status(bvc_cache_adjoint_workspace_size_impl(g, opts, min_bytes, full_bytes));
}

static bvc_status bvc_cache_adjoint_impl(bvc_geometry g, const bvc_function* ffn, const bvc_cache_opts* opts,
                                        const bvc_cache* cache, const double* adj_u, const double* adj_q,
                                        const double* adj_src, double* grad_gv, double* grad_amp, void* workspace,
                                        size_t workspace_bytes, bvc_stream stream) {
  if (g == nullptr || opts == nullptr || cache == nullptr || adj_u == nullptr || adj_q == nullptr ||
      grad_gv == nullptr || workspace == nullptr)
    return BVC_ERR_INVALID_ARG;
  const int D = g->dim;
  const int64_t N = opts->n_samples;
  const int32_t W = opts->walks_per_sample;
  if (cache->dim != D || cache->n != N || cache->z == nullptr || cache->nrm == nullptr ||
      !valid_walk_args((float)opts->eps, opts->max_steps, W))
    return BVC_ERR_INVALID_ARG;
  if (!diff_source_ok(ffn, D) || cache->sigma != 0.0 || opts->sigma != 0.0) return BVC_ERR_UNSUPPORTED;
  const bool has_f = ffn != nullptr && ffn->n_terms > 0;
  if (has_f && grad_amp == nullptr) return BVC_ERR_INVALID_ARG;
  WalkParams P{};
  P.G = g->dev;
  P.chunk = g->tune_chunk;
  P.blocks_per_sm = g->tune_blocks_per_sm;
  if (!make_dev_function(ffn, D, &P.f)) return BVC_ERR_INVALID_ARG;
  const size_t per = ws_per_start(D, W, 0);
  int64_t chunk = ws_chunk(workspace_bytes, per);
  if (chunk < 1) return BVC_ERR_WORKSPACE;
  if (chunk > N) chunk = N;
  cudaStream_t s = (cudaStream_t)stream;
  P.starts = cache->z;
  P.nrm = cache->nrm;
  P.pt_stride = N;
  P.W = W;
  P.eps = (float)opts->eps;
  P.max_steps = opts->max_steps;
  P.seed = opts->seed;
  P.tag = 0;
  P.counter = (unsigned long long*)workspace;
  P.adj_u = adj_u;
  P.adj_q = adj_q;
  P.grad_gv = grad_gv;
  P.grad_amp = grad_amp;
  for (int64_t i0 = 0; i0 < N; i0 += chunk) {
    const int64_t c = (N - i0) < chunk ? (N - i0) : chunk;
    P.i0 = i0;
    P.total = c * (int64_t)W;
    P.wid0 = opts->walk_id_base + (uint64_t)i0 * (uint64_t)W;
    float* fh = ws_first(workspace);
    P.rec = ws_records(workspace, c, D);
    P.first = fh;
    bvc_status st = launch_first_hits(D, g->dev, P.starts, N, i0, c, fh, s);
    if (st != BVC_OK) return st;
    st = launch_walk(D, has_f, kRecAdj, false, P, s);
    if (st != BVC_OK) return st;
    int64_t blocks = (c * 32 + 255) / 256;
    const int64_t cap = (int64_t)num_sms() * 16;
    if (blocks > cap) blocks = cap;
    ProfScope ps("adjoint_cv", s);
    k_adj_cv<<<(unsigned)blocks, 256, 0, s>>>(P.rec, c, W, P.starts, N, i0, fh, g->dev, D, grad_gv);
    BVC_LAUNCH_CHECK();
  }
  if (has_f && cache->n_src_cand > 0 && adj_src != nullptr)
    return bvc_source_adjoint(g, ffn, cache, adj_src, grad_amp, stream);
  return BVC_OK;
}
extern "C" bvc_status bvc_cache_adjoint(bvc_geometry g, const bvc_function* ffn, const bvc_cache_opts* opts,
                                        const bvc_cache* cache, const double* adj_u, const double* adj_q,
                                        const double* adj_src, double* grad_gv, double* grad_amp, void* workspace,
                                        size_t workspace_bytes, bvc_stream stream) {
  return bvc::note_status(bvc_cache_adjoint_impl(g, ffn, opts, cache, adj_u, adj_q, adj_src, grad_gv, grad_amp, workspace, workspace_bytes, stream));
}

// ---------------------------------------------------------------------------
// Walk launch autotuner.  A walk's result depends only on its id, never on
// which thread runs it, so the persistent grid's occupancy and the refill
// chunk change speed only.  bvc_tune_walks samples min(N, 16384) boundary
// points of the caller's problem, and times the cache walks of those points
// (CUDA events on the caller's stream, best of two launches) for resident
// blocks per SM from the maximum down to half of it and refill chunks of
// 64, 128 and 256 walks; the fastest shape is kept in the geometry.
static constexpr int64_t kTuneSamples = 16384;

static int64_t tune_samples(const bvc_cache_opts* o) {
  return o->n_samples < kTuneSamples ? o->n_samples : kTuneSamples;
}

static bvc_status bvc_tune_walks_workspace_size_impl(bvc_geometry g, const bvc_cache_opts* opts, size_t* bytes) {
  if (g == nullptr || opts == nullptr || bytes == nullptr || opts->n_samples < 1 || opts->walks_per_sample < 1)
    return BVC_ERR_INVALID_ARG;
  const int64_t n = tune_samples(opts);
  const size_t pts = (((size_t)n * (2 * g->dim + 1) * sizeof(float)) + 255) & ~size_t(255);
  *bytes = pts + 2 * kWsHead + ws_per_start(g->dim, opts->walks_per_sample, 1) * (size_t)n;
  return BVC_OK;
}
extern "C" bvc_status bvc_tune_walks_workspace_size(bvc_geometry g, const bvc_cache_opts* opts, size_t* bytes) {
  return bvc::note_status(bvc_tune_walks_workspace_size_impl(g, opts, bytes));
}

static bvc_status bvc_geometry_set_walk_shape_impl(bvc_geometry g, int32_t blocks_per_sm, int32_t chunk) {
  if (g == nullptr || blocks_per_sm < 0 || chunk < 0 || chunk > (1 << 20)) return BVC_ERR_INVALID_ARG;
  g->tune_blocks_per_sm = blocks_per_sm;
  g->tune_chunk = chunk;
  return BVC_OK;
}
extern "C" bvc_status bvc_geometry_set_walk_shape(bvc_geometry g, int32_t blocks_per_sm, int32_t chunk) {
  return bvc::note_status(bvc_geometry_set_walk_shape_impl(g, blocks_per_sm, chunk));
}

static bvc_status bvc_tune_walks_impl(bvc_geometry g, const bvc_function* gfn, const bvc_function* ffn,
                                     const bvc_cache_opts* opts, void* workspace, size_t workspace_bytes,
                                     bvc_stream stream, int32_t shape[2], float* best_ms) {
  size_t need = 0;
  bvc_status st = bvc_tune_walks_workspace_size(g, opts, &need);
  if (st != BVC_OK) return st;
  if (workspace == nullptr || !valid_walk_args((float)opts->eps, opts->max_steps, opts->walks_per_sample))
    return BVC_ERR_INVALID_ARG;
  if (workspace_bytes < need) return BVC_ERR_WORKSPACE;
  const int D = g->dim;
  const int64_t n = tune_samples(opts);
  const int32_t W = opts->walks_per_sample;
  cudaStream_t s = (cudaStream_t)stream;
  float* z = (float*)workspace;
  float* nrm = z + (size_t)D * n;
  float* jac = nrm + (size_t)D * n;
  void* ws = (char*)workspace + ((((size_t)n * (2 * D + 1) * sizeof(float)) + 255) & ~size_t(255));
  st = launch_sample_boundary(g, n, opts->offset_l, opts->seed, z, nrm, jac, nullptr, n, s, nullptr);
  if (st != BVC_OK) return st;
  WalkParams P{};
  P.G = g->dev;
  if (!make_dev_function(gfn, D, &P.g) || !make_dev_function(ffn, D, &P.f)) return BVC_ERR_INVALID_ARG;
  P.starts = z;
  P.nrm = nrm;
  P.pt_stride = n;
  P.i0 = 0;
  P.W = W;
  P.total = n * (int64_t)W;
  P.wid0 = opts->walk_id_base;
  P.eps = (float)opts->eps;
  P.max_steps = opts->max_steps;
  P.seed = opts->seed;
  P.tag = 0;
  P.counter = (unsigned long long*)ws;
  float* fh = ws_first(ws);
  P.rec = ws_records(ws, n, D);
  P.first = fh;
  st = launch_first_hits(D, g->dev, z, n, 0, n, fh, s);
  if (st != BVC_OK) return st;
  const bool has_f = P.f.n_terms > 0;
  const int maxb = max_blocks_per_sm(pick_walk(D, has_f, kRecGn, false), kWalkBlock, 0);
  cudaEvent_t e0, e1;
  BVC_CUDA_TRY(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return BVC_ERR_CUDA;
  }
  float best = 3.0e38f;
  int best_b = 0, best_c = 0;
  const int chunks[3] = {64, 128, 256};
  st = BVC_OK;
  for (int b = maxb; b >= (maxb + 1) / 2 && st == BVC_OK; --b)
    for (int ci = 0; ci < 3 && st == BVC_OK; ++ci) {
      P.blocks_per_sm = b;
      P.chunk = chunks[ci];
      float t = 3.0e38f;
      for (int rep = 0; rep < 2 && st == BVC_OK; ++rep) {
        if (cudaEventRecord(e0, s) != cudaSuccess) st = BVC_ERR_CUDA;
        if (st == BVC_OK) st = launch_walk(D, has_f, kRecGn, false, P, s);
        if (st == BVC_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
          st = BVC_ERR_CUDA;
        float ms = 0.0f;
        if (st == BVC_OK && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms < t) t = ms;
      }
      if (st == BVC_OK && t < best) {
        best = t;
        best_b = b;
        best_c = chunks[ci];
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != BVC_OK) {
    (void)cudaGetLastError();
    return st;
  }
  g->tune_blocks_per_sm = best_b;
  g->tune_chunk = best_c;
  if (shape) {
    shape[0] = best_b;
    shape[1] = best_c;
  }
  if (best_ms) *best_ms = best;
  return BVC_OK;
}
extern "C" bvc_status bvc_tune_walks(bvc_geometry g, const bvc_function* gfn, const bvc_function* ffn,
                                     const bvc_cache_opts* opts, void* workspace, size_t workspace_bytes,
                                     bvc_stream stream, int32_t shape[2], float* best_ms) {
  return bvc::note_status(bvc_tune_walks_impl(g, gfn, ffn, opts, workspace, workspace_bytes, stream, shape, best_ms));
}

namespace bvc {
bvc_status walk_points_u(bvc_geometry g, const bvc_function* gfn, const bvc_function* ffn, double sigma,
                         const float* starts, int64_t pt_stride, int64_t i0, int64_t c, int32_t W, float eps,
                         int32_t max_steps, uint64_t seed, uint32_t tag, uint64_t wid0, void* ws, size_t ws_bytes,
                         cudaStream_t s) {
  const int D = g->dim;
  if (!valid_walk_args(eps, max_steps, W) || !(sigma >= 0.0)) return BVC_ERR_INVALID_ARG;
  if (ws_chunk(ws_bytes, ws_per_start(D, W, D)) < c) return BVC_ERR_WORKSPACE;
  WalkParams P{};
  P.G = g->dev;
  P.chunk = g->tune_chunk;
  P.blocks_per_sm = g->tune_blocks_per_sm;
  if (!make_dev_function(gfn, D, &P.g) || !make_dev_function(ffn, D, &P.f)) return BVC_ERR_INVALID_ARG;
  P.starts = starts;
  P.nrm = nullptr;
  P.pt_stride = pt_stride;
  P.W = W;
  P.eps = eps;
  P.max_steps = max_steps;
  P.seed = seed;
  P.tag = tag;
  P.sqs = (float)std::sqrt(sigma);
  P.counter = (unsigned long long*)ws;
  P.i0 = i0;
  P.total = c * (int64_t)W;
  P.wid0 = wid0;
  float* fh = ws_first(ws);
  P.rec = ws_records(ws, c, D);
  P.first = fh;
  bvc_status st = launch_first_hits(D, g->dev, starts, pt_stride, i0, c, fh, s);
  if (st != BVC_OK) return st;
  return launch_walk(D, P.f.n_terms > 0, kRecGrad, false, P, s);
}

const float* walk_records_u(void* ws, int64_t c, int dim) { return ws_records(ws, c, dim); }
}  // namespace bvc

static bvc_status wos_estimate_workspace_size_impl(int32_t dim, int64_t m, int32_t walks, size_t* min_bytes,
                                                  size_t* full_bytes) {
  if ((dim != 2 && dim != 3) || m < 0 || walks < 1) return BVC_ERR_INVALID_ARG;
  const size_t per_pt = ws_per_start(dim, walks, dim);
  if (min_bytes) *min_bytes = 2 * kWsHead + per_pt;
  if (full_bytes) *full_bytes = 2 * kWsHead + per_pt * (size_t)m;
  return BVC_OK;
}
extern "C" bvc_status wos_estimate_workspace_size(int32_t dim, int64_t m, int32_t walks, size_t* min_bytes,
                                                  size_t* full_bytes) {
  return bvc::note_status(wos_estimate_workspace_size_impl(dim, m, walks, min_bytes, full_bytes));
}

__global__ void k_add_walk_count(int64_t* counts, int64_t w) {
  if (threadIdx.x == 0 && blockIdx.x == 0) counts[0] += w;
}

static bvc_status wos_estimate_sigma_impl(bvc_geometry g, const bvc_function* gfn, const bvc_function* ffn,
                                         double sigma, bvc_eval_state* state, int32_t walks, float eps,
                                         int32_t max_steps, uint64_t seed, uint64_t id_base, void* workspace,
                                         size_t workspace_bytes, bvc_stream stream) {
  if (g == nullptr || state == nullptr || state->dim != g->dim || state->m < 0 || state->counts == nullptr ||
      !valid_walk_args(eps, max_steps, walks) || !std::isfinite(sigma) || sigma < 0.0)
    return BVC_ERR_INVALID_ARG;
  const int64_t m = state->m;
  if (m > 0 && (state->x == nullptr || state->u_bnd == nullptr || workspace == nullptr)) return BVC_ERR_INVALID_ARG;
  const int D = g->dim;
  WalkParams P{};
  P.G = g->dev;
  P.chunk = g->tune_chunk;
  P.blocks_per_sm = g->tune_blocks_per_sm;
  if (!make_dev_function(gfn, D, &P.g) || !make_dev_function(ffn, D, &P.f)) return BVC_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (m > 0) {
    const size_t per_pt = ws_per_start(D, walks, D);
    int64_t chunk = ws_chunk(workspace_bytes, per_pt);
    if (chunk < 1) return BVC_ERR_WORKSPACE;
    if (chunk > m) chunk = m;
    P.starts = state->x;
    P.nrm = nullptr;
    P.pt_stride = m;
    P.W = walks;
    P.eps = eps;
    P.max_steps = max_steps;
    P.seed = seed;
    P.tag = 3;
    P.sqs = (float)std::sqrt(sigma);
    P.counter = (unsigned long long*)workspace;
    const bool grad = state->grad_bnd != nullptr;
    for (int64_t i0 = 0; i0 < m; i0 += chunk) {
      const int64_t c = (m - i0) < chunk ? (m - i0) : chunk;
      P.i0 = i0;
      P.total = c * (int64_t)walks;
      P.wid0 = id_base + (uint64_t)i0 * (uint64_t)walks;
      float* fh = ws_first(workspace);
      P.rec = ws_records(workspace, c, D);
      P.first = fh;
      bvc_status st = launch_first_hits(D, g->dev, P.starts, m, i0, c, fh, s);
      if (st != BVC_OK) return st;
      st = launch_walk(D, P.f.n_terms > 0, kRecGrad, g->counting != 0, P, s);
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
        for (int a = 0; a < D; ++a) R.out[1 + a] = state->grad_bnd + (int64_t)a * m + i0;
      st = launch_reduce(R, s);
      if (st != BVC_OK) return st;
    }
  }
  {
    ProfScope ps("add_counts", s);
    k_add_walk_count<<<1, 32, 0, s>>>(state->counts, walks);
  }
  BVC_LAUNCH_CHECK();
  return BVC_OK;
}
extern "C" bvc_status wos_estimate_sigma(bvc_geometry g, const bvc_function* gfn, const bvc_function* ffn,
                                         double sigma, bvc_eval_state* state, int32_t walks, float eps,
                                         int32_t max_steps, uint64_t seed, uint64_t id_base, void* workspace,
                                         size_t workspace_bytes, bvc_stream stream) {
  return bvc::note_status(wos_estimate_sigma_impl(g, gfn, ffn, sigma, state, walks, eps, max_steps, seed, id_base, workspace, workspace_bytes, stream));
}

static bvc_status wos_estimate_impl(bvc_geometry g, const bvc_function* gfn, const bvc_function* ffn,
                                   bvc_eval_state* state, int32_t walks, float eps, int32_t max_steps, uint64_t seed,
                                   uint64_t id_base, void* workspace, size_t workspace_bytes, bvc_stream stream) {
  return wos_estimate_sigma(g, gfn, ffn, 0.0, state, walks, eps, max_steps, seed, id_base, workspace,
                            workspace_bytes, stream);
}
extern "C" bvc_status wos_estimate(bvc_geometry g, const bvc_function* gfn, const bvc_function* ffn,
                                   bvc_eval_state* state, int32_t walks, float eps, int32_t max_steps, uint64_t seed,
                                   uint64_t id_base, void* workspace, size_t workspace_bytes, bvc_stream stream) {
  return bvc::note_status(wos_estimate_impl(g, gfn, ffn, state, walks, eps, max_steps, seed, id_base, workspace, workspace_bytes, stream));
}

// ---------------------------------------------------------------------------
// Many right-hand sides (Laplace, f = 0).  With no source term a walk's path
// does not depend on g, so the walks of a cache are run once, recording
// their end points, and every right-hand side g_k = sum_m C[k][m] phi_m
// (phi_m the POLY monomials) is recovered from per-sample moments:
//   mom_u[i][m] = mean_j phi_m(end_ij)
//   mom_q[i][m] = mean_j s_ij (phi_m(end_ij) - phi_m(p0_i))
// where p0_i is the closest point of sample i and s_ij = (d/R0)(n . w0);
// then u^_ik = sum_m C[k][m] mom_u[i][m] and du/dn^_ik likewise -- the same
// estimates the single-RHS walks give, by linearity (each walk's U and
// n.grad are linear in g).
namespace bvc {

template <int D>
struct Mono {
  static constexpr int kN = D == 2 ? 15 : 35;
};

// Exponents of monomial m in the POLY order (degree t, then x power
// descending, then y power descending).
template <int D>
__host__ __device__ constexpr void mono_exp(int m, int& i, int& j, int& k) {
  int idx = 0;
  for (int t = 0; t <= 4; ++t)
    for (int a = t; a >= 0; --a) {
      if (D == 2) {
        if (idx == m) {
          i = a;
          j = t - a;
          k = 0;
          return;
        }
        ++idx;
      } else {
        for (int b = t - a; b >= 0; --b) {
          if (idx == m) {
            i = a;
            j = b;
            k = t - a - b;
            return;
          }
          ++idx;
        }
      }
    }
  i = j = k = 0;
}

template <int D>
__device__ __forceinline__ void powers(const float* p, float (&xp)[5], float (&yp)[5], float (&zp)[5]) {
  xp[0] = yp[0] = zp[0] = 1.0f;
#pragma unroll
  for (int e = 1; e < 5; ++e) {
    xp[e] = xp[e - 1] * p[0];
    yp[e] = yp[e - 1] * p[1];
    zp[e] = D == 3 ? zp[e - 1] * p[D - 1] : 0.0f;
  }
}

template <int D, int M>
__device__ __forceinline__ float mono(const float (&xp)[5], const float (&yp)[5], const float (&zp)[5]) {
  constexpr int i = []() { int a = 0, b = 0, c = 0; mono_exp<D>(M, a, b, c); return a; }();
  constexpr int j = []() { int a = 0, b = 0, c = 0; mono_exp<D>(M, a, b, c); return b; }();
  constexpr int k = []() { int a = 0, b = 0, c = 0; mono_exp<D>(M, a, b, c); return c; }();
  return D == 2 ? xp[i] * yp[j] : xp[i] * yp[j] * zp[k];
}

template <int D, int M, int NM>
struct MonoLoop {
  __device__ __forceinline__ static void acc(const float (&xp)[5], const float (&yp)[5], const float (&zp)[5],
                                             const float (&x0)[5], const float (&y0)[5], const float (&z0)[5],
                                             float sj, float* au, float* aq) {
    const float ph = mono<D, M>(xp, yp, zp);
    au[M] += ph;
    aq[M] = fmaf(sj, ph - mono<D, M>(x0, y0, z0), aq[M]);
    MonoLoop<D, M + 1, NM>::acc(xp, yp, zp, x0, y0, z0, sj, au, aq);
  }
};
template <int D, int NM>
struct MonoLoop<D, NM, NM> {
  __device__ __forceinline__ static void acc(const float (&)[5], const float (&)[5], const float (&)[5],
                                             const float (&)[5], const float (&)[5], const float (&)[5], float,
                                             float*, float*) {}
};

// One warp per sample: FP32 partials per lane over its walks, FP64
// fixed-order warp sums.
template <int D>
__global__ void __launch_bounds__(256) k_moments(const float* __restrict__ rec, int64_t c, int32_t W,
                                                 const float* __restrict__ starts, int64_t pt_stride, int64_t i0,
                                                 const float* __restrict__ fh, double* __restrict__ mom_u,
                                                 double* __restrict__ mom_q) {
  constexpr int NM = Mono<D>::kN;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t total = c * (int64_t)W;
  for (int64_t r = warp; r < c; r += nwarps) {
    float p0[D];
#pragma unroll
    for (int a = 0; a < D; ++a) p0[a] = starts[a * pt_stride + i0 + r] - fh[(1 + a) * c + r];
    float x0[5], y0[5], z0[5];
    powers<D>(p0, x0, y0, z0);
    float au[NM], aq[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) au[m] = aq[m] = 0.0f;
    for (int j = lane; j < W; j += 32) {
      const int64_t t = r * W + j;
      float pe[D];
#pragma unroll
      for (int a = 0; a < D; ++a) pe[a] = rec[a * total + t];
      const float sj = rec[D * total + t];
      float xp[5], yp[5], zp[5];
      powers<D>(pe, xp, yp, zp);
      MonoLoop<D, 0, NM>::acc(xp, yp, zp, x0, y0, z0, sj, au, aq);
    }
#pragma unroll
    for (int m = 0; m < NM; ++m) {
      double su = (double)au[m], sq = (double)aq[m];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        su += __shfl_xor_sync(0xffffffffu, su, o);
        sq += __shfl_xor_sync(0xffffffffu, sq, o);
      }
      if (lane == 0) {
        mom_u[(i0 + r) * NM + m] = su / (double)W;
        mom_q[(i0 + r) * NM + m] = sq / (double)W;
      }
    }
  }
}

// Per sample, the walk means of the per-bump source records (the end-point
// walks' planes D + 1 .. D + 2 kMaxBumps): FP32 partials per lane over its
// walks, FP64 fixed-order warp sums, as k_moments.
__global__ void __launch_bounds__(256) k_src_moments(const float* __restrict__ rec, int64_t c, int32_t W, int32_t D,
                                                     int64_t i0, double* __restrict__ mom_su,
                                                     double* __restrict__ mom_sq) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t total = c * (int64_t)W;
  const float* ru = rec + (int64_t)(D + 1) * total;
  const float* rq = rec + (int64_t)(D + 1 + kMaxBumps) * total;
  for (int64_t r = warp; r < c; r += nwarps) {
    float au[kMaxBumps], aq[kMaxBumps];
#pragma unroll
    for (int b = 0; b < kMaxBumps; ++b) au[b] = aq[b] = 0.0f;
    for (int j = lane; j < W; j += 32) {
      const int64_t t = r * W + j;
#pragma unroll
      for (int b = 0; b < kMaxBumps; ++b) {
        au[b] += ru[b * total + t];
        aq[b] += rq[b * total + t];
      }
    }
#pragma unroll
    for (int b = 0; b < kMaxBumps; ++b) {
      double su = (double)au[b], sq = (double)aq[b];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        su += __shfl_xor_sync(0xffffffffu, su, o);
        sq += __shfl_xor_sync(0xffffffffu, sq, o);
      }
      if (lane == 0) {
        mom_su[(i0 + r) * kMaxBumps + b] = su / (double)W;
        mom_sq[(i0 + r) * kMaxBumps + b] = sq / (double)W;
      }
    }
  }
}

// Per sample: u^_k, du/dn^_k for every right-hand side (FP64) and the
// gather tiles, grouped by BVC_MULTI_GROUP right-hand sides:
// [group][sample][8 + 2 G] floats = z (4), n (4), a_k (G), b_k (G) with
// 1/p = |dOmega| jac (the sample's offset element, Sec. 3.2) and
//   2D  a = u^ /(2 pi p),  b = -du/dn^ /(2 pi p) ln2/2   (u += a (n.d)/r^2 + b lg2 r^2)
//   3D  a = u^ /(4 pi p),  b = du/dn^ /(4 pi p)          (u += a (n.d)/r^3 + b/r)
// With a source (B > 0 bumps) each coefficient row holds NM + B values and
// the source moments add sum_b A[k][b] mom_s?[i][b]; rows_g is the number
// of rows of each group's tile block (n, plus the source candidates).
template <int D>
__global__ void __launch_bounds__(128) k_project(const double* __restrict__ C, int32_t K, int64_t n,
                                                 const double* __restrict__ mom_u, const double* __restrict__ mom_q,
                                                 int32_t B, const double* __restrict__ mom_su,
                                                 const double* __restrict__ mom_sq, int64_t rows_g,
                                                 const float* __restrict__ z, const float* __restrict__ nrm,
                                                 const float* __restrict__ jac, double meas,
                                                 double* __restrict__ u_hat,
                                                 double* __restrict__ q_hat, float* __restrict__ packed,
                                                 const int32_t* __restrict__ sample_mesh,
                                                 const BatchMeshDev* __restrict__ meshes) {
  constexpr int NM = Mono<D>::kN;
  constexpr int G = BVC_MULTI_GROUP;
  constexpr int S = 8 + 2 * G;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int CS = NM + B;  // coefficient row length
  double mu[NM], mq[NM];
#pragma unroll
  for (int m = 0; m < NM; ++m) {
    mu[m] = mom_u[i * NM + m];
    mq[m] = mom_q[i * NM + m];
  }
  if (sample_mesh != nullptr) {  // a batch: this sample's mesh's coefficients and measure
    const int32_t msh = sample_mesh[i];
    C += (int64_t)msh * K * NM;
    meas = meshes[msh].measure;
  }
  const int groups = (K + G - 1) / G;
  const double ip = meas * (double)jac[i];
  const double ca = D == 2 ? ip / 6.283185307179586476925 : ip / 12.566370614359172953850;
  const double cb = D == 2 ? -ca * 0.34657359027997265471 : ca;
  for (int g = 0; g < groups; ++g) {
    float* row = packed + ((int64_t)g * rows_g + i) * S;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      row[a] = a < D ? z[a * n + i] : 0.0f;
      row[4 + a] = a < D ? nrm[a * n + i] : 0.0f;
    }
    for (int s = 0; s < G; ++s) {
      const int k = g * G + s;
      double u = 0.0, q = 0.0;
      if (k < K) {
#pragma unroll
        for (int m = 0; m < NM; ++m) {
          u = fma(C[k * CS + m], mu[m], u);
          q = fma(C[k * CS + m], mq[m], q);
        }
        for (int b = 0; b < B; ++b) {
          u = fma(C[k * CS + NM + b], mom_su[i * kMaxBumps + b], u);
          q = fma(C[k * CS + NM + b], mom_sq[i * kMaxBumps + b], q);
        }
        u_hat[(int64_t)k * n + i] = u;
        q_hat[(int64_t)k * n + i] = q;
      }
      row[8 + s] = (float)(u * ca);
      row[8 + G + s] = (float)(q * cb);
    }
  }
}

// Source candidate rows of the gather tiles, after the n sample rows of each
// group: (y, 0 normal), a_k = 0 and b_k the Eq. 4 weight of right-hand side
// k, c_jk = sum_b A[k][b] |box| psi_b(y_j), scaled so that the gather's 1/n
// over all rows gives 1/M over the candidates:
//   2D  b = (n/M) c/(2 pi) ln2/2  (u += b lg2 r^2)     3D  b = -(n/M) c/(4 pi)  (u += b/r)
template <int D>
__global__ void __launch_bounds__(128) k_project_src(const double* __restrict__ C, int32_t K, int32_t B, int64_t n,
                                                     int64_t M, const int64_t* __restrict__ kept,
                                                     const float* __restrict__ src_y,
                                                     const float* __restrict__ src_psi, float* __restrict__ packed) {
  constexpr int NM = Mono<D>::kN;
  constexpr int G = BVC_MULTI_GROUP;
  constexpr int S = 8 + 2 * G;
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= M || j >= *kept) return;
  const int CS = NM + B;
  const double scale = D == 2 ? (double)n / (double)M / 6.283185307179586476925 * 0.34657359027997265471
                              : -(double)n / (double)M / 12.566370614359172953850;
  double psi[kMaxBumps];
#pragma unroll
  for (int b = 0; b < kMaxBumps; ++b) psi[b] = (double)src_psi[j * kMaxBumps + b];
  const int groups = (K + G - 1) / G;
  for (int g = 0; g < groups; ++g) {
    float* row = packed + ((int64_t)g * (n + M) + n + j) * S;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      row[a] = a < D ? src_y[a * M + j] : 0.0f;
      row[4 + a] = 0.0f;
    }
    for (int s = 0; s < G; ++s) {
      const int k = g * G + s;
      double c = 0.0;
      if (k < K)
        for (int b = 0; b < B; ++b) c = fma(C[k * CS + NM + b], psi[b], c);
      row[8 + s] = 0.0f;
      row[8 + G + s] = (float)(c * scale);
    }
  }
}

// |box| psi_b(y_j) of the kept candidates (psi_b the shape's bumps).
template <int D>
__global__ void __launch_bounds__(256) k_src_psi(DevFunction shape, const float* __restrict__ src_y, int64_t M,
                                                 const int64_t* __restrict__ kept, double box,
                                                 float* __restrict__ src_psi) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= M || j >= *kept) return;
  float y[D];
#pragma unroll
  for (int a = 0; a < D; ++a) y[a] = src_y[a * M + j];
  float psi[kMaxBumps];
  bump_shapes<D>(shape, y, psi);
#pragma unroll
  for (int b = 0; b < kMaxBumps; ++b) src_psi[j * kMaxBumps + b] = (float)((double)psi[b] * box);
}

}  // namespace bvc

static bool valid_multi(const bvc_multi_cache* c, int dim) {
  if (!(c != nullptr && c->dim == dim && c->n >= 1 && c->k >= 1 && c->z && c->nrm && c->jac && c->mom_u && c->mom_q &&
        c->u_hat && c->dudn_hat && c->packed))
    return false;
  if (c->n_bumps < 0 || c->n_bumps > kMaxBumps || c->n_src_cand < 0) return false;
  if (c->n_bumps > 0 && (c->mom_su == nullptr || c->mom_sq == nullptr)) return false;
  if (c->n_src_cand > 0 && (c->n_bumps == 0 || !c->src_y || !c->src_psi || !c->n_src_dev)) return false;
  return true;
}

static bvc_status launch_project(const double* coeffs, bvc_multi_cache* c, cudaStream_t s,
                                 const int32_t* sample_mesh = nullptr, const BatchMeshDev* meshes = nullptr) {
  const unsigned grid = (unsigned)((c->n + 127) / 128);
  const int32_t B = c->n_bumps;
  const int64_t M = c->n_src_cand, rows = c->n + M;
  ProfScope ps("multi_project", s);
  if (c->dim == 2)
    k_project<2><<<grid, 128, 0, s>>>(coeffs, c->k, c->n, c->mom_u, c->mom_q, B, c->mom_su, c->mom_sq, rows, c->z,
                                      c->nrm, c->jac, c->bnd_measure, c->u_hat, c->dudn_hat, c->packed, sample_mesh,
                                      meshes);
  else
    k_project<3><<<grid, 128, 0, s>>>(coeffs, c->k, c->n, c->mom_u, c->mom_q, B, c->mom_su, c->mom_sq, rows, c->z,
                                      c->nrm, c->jac, c->bnd_measure, c->u_hat, c->dudn_hat, c->packed, sample_mesh,
                                      meshes);
  if (M > 0) {
    const unsigned gs = (unsigned)((M + 127) / 128);
    if (c->dim == 2)
      k_project_src<2><<<gs, 128, 0, s>>>(coeffs, c->k, B, c->n, M, c->n_src_dev, c->src_y, c->src_psi, c->packed);
    else
      k_project_src<3><<<gs, 128, 0, s>>>(coeffs, c->k, B, c->n, M, c->n_src_dev, c->src_y, c->src_psi, c->packed);
  }
  BVC_LAUNCH_CHECK();
  return BVC_OK;
}

// End-point walks of every start of a multi-RHS cache (one mesh, or a batch
// when E.sample_mesh is set), in chunks that fit the workspace: first
// closest-point queries, the walks, and the per-sample monomial moments.
struct EndWalks {
  DevGeometry G;
  int dim;
  bool counting;
  int32_t W;
  float eps;
  int32_t max_steps;
  uint64_t seed, wid_base;
  const int32_t* sample_mesh;
  const BatchMeshDev* meshes;
  const uint64_t* seed_dev;
  bool src;       // a bump source: per-bump records and their moments
  DevFunction f;  // its shape (src only)
};

static bvc_status run_end_walks(const EndWalks& E, bvc_multi_cache* cache, void* workspace, int64_t chunk,
                                cudaStream_t s) {
  const int D = E.dim;
  const int64_t N = cache->n;
  WalkParams P{};
  P.G = E.G;
  P.starts = cache->z;
  P.nrm = cache->nrm;
  P.pt_stride = N;
  P.W = E.W;
  P.eps = E.eps;
  P.max_steps = E.max_steps;
  P.seed = E.seed;
  P.tag = 0;
  P.counter = (unsigned long long*)workspace;
  P.sample_mesh = E.sample_mesh;
  P.meshes = E.meshes;
  P.seed_dev = E.seed_dev;
  if (E.src) P.f = E.f;
  for (int64_t i0 = 0; i0 < N; i0 += chunk) {
    const int64_t c = (N - i0) < chunk ? (N - i0) : chunk;
    P.i0 = i0;
    P.total = c * (int64_t)E.W;
    P.wid0 = E.wid_base + (uint64_t)i0 * (uint64_t)E.W;
    float* fh = ws_first(workspace);
    P.rec = ws_records(workspace, c, D);
    P.first = fh;
    bvc_status st = launch_first_hits(D, E.G, P.starts, N, i0, c, fh, s, E.sample_mesh, E.meshes);
    if (st != BVC_OK) return st;
    st = launch_walk(D, E.src, kRecEnd, E.counting, P, s);
    if (st != BVC_OK) return st;
    int64_t blocks = (c * 32 + 255) / 256;
    const int64_t cap = (int64_t)num_sms() * 16;
    if (blocks > cap) blocks = cap;
    ProfScope ps("multi_moments", s);
    if (D == 2)
      k_moments<2><<<(unsigned)blocks, 256, 0, s>>>(P.rec, c, E.W, P.starts, N, i0, fh, cache->mom_u, cache->mom_q);
    else
      k_moments<3><<<(unsigned)blocks, 256, 0, s>>>(P.rec, c, E.W, P.starts, N, i0, fh, cache->mom_u, cache->mom_q);
    if (E.src)
      k_src_moments<<<(unsigned)blocks, 256, 0, s>>>(P.rec, c, E.W, D, i0, cache->mom_su, cache->mom_sq);
    BVC_LAUNCH_CHECK();
  }
  return BVC_OK;
}

extern "C" int32_t bvc_poly_terms(int32_t dim) { return dim == 2 ? 15 : (dim == 3 ? 35 : 0); }

static bvc_status bvc_multi_cache_build_workspace_size_impl(bvc_geometry g, int64_t n, int32_t walks,
                                                           size_t* min_bytes, size_t* full_bytes) {
  if (g == nullptr || n < 1 || walks < 1) return BVC_ERR_INVALID_ARG;
  const size_t per = ws_per_start(g->dim, walks, g->dim);
  if (min_bytes) *min_bytes = 2 * kWsHead + per;
  if (full_bytes) *full_bytes = 2 * kWsHead + per * (size_t)n;
  return BVC_OK;
}
extern "C" bvc_status bvc_multi_cache_build_workspace_size(bvc_geometry g, int64_t n, int32_t walks,
                                                           size_t* min_bytes, size_t* full_bytes) {
  return bvc::note_status(bvc_multi_cache_build_workspace_size_impl(g, n, walks, min_bytes, full_bytes));
}

static bvc_status bvc_multi_cache_build_impl(bvc_geometry g, const double* coeffs, const bvc_cache_opts* opts,
                                            bvc_multi_cache* cache, void* workspace, size_t workspace_bytes,
                                            bvc_stream stream) {
  if (g == nullptr || opts == nullptr || coeffs == nullptr || workspace == nullptr || cache == nullptr)
    return BVC_ERR_INVALID_ARG;
  const int D = g->dim;
  const int64_t N = opts->n_samples;
  const int32_t W = opts->walks_per_sample;
  if (cache->n_src_cand != 0) return BVC_ERR_INVALID_ARG;  // a source cache: bvc_multi_cache_build_source
  cache->n_bumps = 0;
  if (!valid_multi(cache, D) || cache->n != N || !valid_walk_args((float)opts->eps, opts->max_steps, W) ||
      !(opts->offset_l > 0.0))
    return BVC_ERR_INVALID_ARG;
  if (src_candidates(opts, D) != 0 || opts->sigma != 0.0) return BVC_ERR_UNSUPPORTED;  // Laplace (f = 0) only
  const size_t per = ws_per_start(D, W, D);
  int64_t chunk = ws_chunk(workspace_bytes, per);
  if (chunk < 1) return BVC_ERR_WORKSPACE;
  if (chunk > N) chunk = N;
  cudaStream_t s = (cudaStream_t)stream;
  cache->bnd_measure = g->measure;
  bvc_status st =
      bvc_sample_boundary(g, N, opts->offset_l, opts->seed, cache->z, cache->nrm, cache->jac, nullptr, stream);
  if (st != BVC_OK) return st;
  EndWalks E{};
  E.G = g->dev;
  E.dim = D;
  E.counting = g->counting != 0;
  E.W = W;
  E.eps = (float)opts->eps;
  E.max_steps = opts->max_steps;
  E.seed = opts->seed;
  E.wid_base = opts->walk_id_base;
  st = run_end_walks(E, cache, workspace, chunk, s);
  if (st != BVC_OK) return st;
  return launch_project(coeffs, cache, s);
}
extern "C" bvc_status bvc_multi_cache_build(bvc_geometry g, const double* coeffs, const bvc_cache_opts* opts,
                                            bvc_multi_cache* cache, void* workspace, size_t workspace_bytes,
                                            bvc_stream stream) {
  return bvc::note_status(bvc_multi_cache_build_impl(g, coeffs, opts, cache, workspace, workspace_bytes, stream));
}

// The source variant: records D + 1 + 2 kMaxBumps planes per walk; the
// source candidates' sampling scratch follows in the same workspace (used
// after the walks).
static size_t multi_src_scratch(int64_t ncand) {
  size_t b = 0;
  bvc_sample_source_workspace_size(ncand, &b);
  return b + ((size_t)ncand * 8 + 255) / 256 * 256;  // + the candidates' f(y) |box| (unused)
}
static bvc_status bvc_multi_cache_build_source_workspace_size_impl(bvc_geometry g, const bvc_cache_opts* opts,
                                                                  size_t* min_bytes, size_t* full_bytes) {
  if (g == nullptr || opts == nullptr || opts->n_samples < 1 || opts->walks_per_sample < 1) return BVC_ERR_INVALID_ARG;
  const int64_t ncand = src_candidates(opts, g->dim);
  if (ncand < 1) return BVC_ERR_INVALID_ARG;
  const size_t per = ws_per_start(g->dim, opts->walks_per_sample, g->dim + 2 * kMaxBumps);
  const size_t src = multi_src_scratch(ncand);
  if (min_bytes) *min_bytes = std::max(2 * kWsHead + per, src);
  if (full_bytes) *full_bytes = std::max(2 * kWsHead + per * (size_t)opts->n_samples, src);
  return BVC_OK;
}
extern "C" bvc_status bvc_multi_cache_build_source_workspace_size(bvc_geometry g, const bvc_cache_opts* opts,
                                                                  size_t* min_bytes, size_t* full_bytes) {
  return bvc::note_status(bvc_multi_cache_build_source_workspace_size_impl(g, opts, min_bytes, full_bytes));
}

static bvc_status bvc_multi_cache_build_source_impl(bvc_geometry g, const bvc_function* shape, const double* coeffs,
                                                   const bvc_cache_opts* opts, bvc_multi_cache* cache,
                                                   void* workspace, size_t workspace_bytes, bvc_stream stream) {
  if (g == nullptr || opts == nullptr || coeffs == nullptr || workspace == nullptr || shape == nullptr ||
      cache == nullptr)
    return BVC_ERR_INVALID_ARG;
  const int D = g->dim;
  const int64_t N = opts->n_samples;
  const int32_t W = opts->walks_per_sample;
  const int64_t ncand = src_candidates(opts, D);
  if (opts->src_grid[0] < 1 || opts->src_grid[1] < 1 || (D == 3 && opts->src_grid[2] < 1)) return BVC_ERR_INVALID_ARG;
  if (shape->n_terms != 1 || (shape->terms[0].kind != BVC_FN_GAUSS && shape->terms[0].kind != BVC_FN_GAUSS_LAPLACIAN))
    return BVC_ERR_UNSUPPORTED;
  const int head = shape->terms[0].kind == BVC_FN_GAUSS_LAPLACIAN ? 3 : 1;
  const int nc = shape->terms[0].n_coeffs;
  const int B = (nc - head) / (1 + D);
  if (nc < head + 1 + D || (nc - head) % (1 + D) != 0 || B > kMaxBumps) return BVC_ERR_INVALID_ARG;
  cache->n_bumps = B;
  if (!valid_multi(cache, D) || cache->n != N || cache->n_src_cand != ncand ||
      !valid_walk_args((float)opts->eps, opts->max_steps, W) || !(opts->offset_l > 0.0))
    return BVC_ERR_INVALID_ARG;
  if (opts->sigma != 0.0) return BVC_ERR_UNSUPPORTED;
  DevFunction f;
  if (!make_dev_function(shape, D, &f)) return BVC_ERR_INVALID_ARG;
  const size_t per = ws_per_start(D, W, D + 2 * kMaxBumps);
  int64_t chunk = ws_chunk(workspace_bytes, per);
  if (chunk < 1 || workspace_bytes < multi_src_scratch(ncand)) return BVC_ERR_WORKSPACE;
  if (chunk > N) chunk = N;
  cudaStream_t s = (cudaStream_t)stream;
  cache->bnd_measure = g->measure;
  bvc_status st =
      bvc_sample_boundary(g, N, opts->offset_l, opts->seed, cache->z, cache->nrm, cache->jac, nullptr, stream);
  if (st != BVC_OK) return st;
  EndWalks E{};
  E.G = g->dev;
  E.dim = D;
  E.counting = g->counting != 0;
  E.W = W;
  E.eps = (float)opts->eps;
  E.max_steps = opts->max_steps;
  E.seed = opts->seed;
  E.wid_base = opts->walk_id_base;
  E.src = true;
  E.f = f;
  st = run_end_walks(E, cache, workspace, chunk, s);
  if (st != BVC_OK) return st;
  // Eq. 4's candidates, as bvc_cache_build samples them (the shape's f(y)
  // |box| goes to scratch; the bump values are kept instead)
  size_t sw = 0;
  bvc_sample_source_workspace_size(ncand, &sw);
  bvc_cache tmp{};
  tmp.dim = D;
  tmp.n_src_cand = ncand;
  tmp.src_y = cache->src_y;
  tmp.src_c = (double*)((char*)workspace + sw);
  tmp.n_src_dev = cache->n_src_dev;
  st = bvc_sample_source(g, shape, opts->src_grid, opts->seed, opts->offset_l, &tmp, workspace, sw, stream);
  if (st != BVC_OK) return st;
  double box = 1.0;
  for (int a = 0; a < D; ++a) box *= (double)g->hi[a] - (double)g->lo[a];
  {
    ProfScope ps("multi_source_psi", s);
    const unsigned gs = (unsigned)((ncand + 255) / 256);
    if (D == 2)
      k_src_psi<2><<<gs, 256, 0, s>>>(f, cache->src_y, ncand, cache->n_src_dev, box, cache->src_psi);
    else
      k_src_psi<3><<<gs, 256, 0, s>>>(f, cache->src_y, ncand, cache->n_src_dev, box, cache->src_psi);
    BVC_LAUNCH_CHECK();
  }
  return launch_project(coeffs, cache, s);
}
extern "C" bvc_status bvc_multi_cache_build_source(bvc_geometry g, const bvc_function* shape, const double* coeffs,
                                                   const bvc_cache_opts* opts, bvc_multi_cache* cache,
                                                   void* workspace, size_t workspace_bytes, bvc_stream stream) {
  return bvc::note_status(
      bvc_multi_cache_build_source_impl(g, shape, coeffs, opts, cache, workspace, workspace_bytes, stream));
}

static bvc_status bvc_multi_cache_project_impl(const double* coeffs, bvc_multi_cache* cache, bvc_stream stream) {
  if (coeffs == nullptr || cache == nullptr || (cache->dim != 2 && cache->dim != 3) || !valid_multi(cache, cache->dim))
    return BVC_ERR_INVALID_ARG;
  return launch_project(coeffs, cache, (cudaStream_t)stream);
}
extern "C" bvc_status bvc_multi_cache_project(const double* coeffs, bvc_multi_cache* cache, bvc_stream stream) {
  return bvc::note_status(bvc_multi_cache_project_impl(coeffs, cache, stream));
}

// ---------------------------------------------------------------------------
// Batches of meshes: every mesh's K1 into its sample range, then the
// end-point walks of all meshes in one launch per workspace chunk over the
// forest, the moments and one projection with per-mesh coefficients.
static bool valid_batch_cache(const bvc_batch_s* b, const bvc_multi_cache* c) {
  // batches solve Laplace problems: no source part
  return b != nullptr && valid_multi(c, b->dim) && c->n == b->n_total && c->k == b->k && c->n_bumps == 0 &&
         c->n_src_cand == 0;
}

static bvc_status bvc_batch_build_workspace_size_impl(bvc_batch b, size_t* min_bytes, size_t* full_bytes) {
  if (b == nullptr) return BVC_ERR_INVALID_ARG;
  const size_t per = ws_per_start(b->dim, b->walks, b->dim);
  if (min_bytes) *min_bytes = 2 * kWsHead + per;
  if (full_bytes) *full_bytes = 2 * kWsHead + per * (size_t)b->n_total;
  return BVC_OK;
}
extern "C" bvc_status bvc_batch_build_workspace_size(bvc_batch b, size_t* min_bytes, size_t* full_bytes) {
  return bvc::note_status(bvc_batch_build_workspace_size_impl(b, min_bytes, full_bytes));
}

static bvc_status bvc_batch_build_impl(bvc_batch b, const double* coeffs, const uint64_t* seed, bvc_multi_cache* cache,
                                      void* workspace, size_t workspace_bytes, bvc_stream stream) {
  if (coeffs == nullptr || seed == nullptr || workspace == nullptr || !valid_batch_cache(b, cache))
    return BVC_ERR_INVALID_ARG;
  const size_t per = ws_per_start(b->dim, b->walks, b->dim);
  int64_t chunk = ws_chunk(workspace_bytes, per);
  if (chunk < 1) return BVC_ERR_WORKSPACE;
  if (chunk > b->n_total) chunk = b->n_total;
  cudaStream_t s = (cudaStream_t)stream;
  cache->bnd_measure = 0.0;
  for (int j = 0; j < b->count; ++j) {
    const BatchMeshDev& m = b->mesh[j];
    const bvc_status st =
        launch_sample_boundary(b->geoms[j], m.n_smp, b->offset_l[j], 0, cache->z + m.smp_off, cache->nrm + m.smp_off,
                               cache->jac + m.smp_off, nullptr, b->n_total, s, seed);
    if (st != BVC_OK) return st;
  }
  EndWalks E{};
  E.G = b->forest;
  E.dim = b->dim;
  E.counting = b->counting != 0;
  E.W = b->walks;
  E.eps = b->mesh[0].eps;
  E.max_steps = b->max_steps;
  E.seed = 0;
  E.seed_dev = seed;
  E.wid_base = 0;
  E.sample_mesh = b->sample_mesh;
  E.meshes = b->table;
  const bvc_status st = run_end_walks(E, cache, workspace, chunk, s);
  if (st != BVC_OK) return st;
  return launch_project(coeffs, cache, s, b->sample_mesh, b->table);
}
extern "C" bvc_status bvc_batch_build(bvc_batch b, const double* coeffs, const uint64_t* seed, bvc_multi_cache* cache,
                                      void* workspace, size_t workspace_bytes, bvc_stream stream) {
  return bvc::note_status(bvc_batch_build_impl(b, coeffs, seed, cache, workspace, workspace_bytes, stream));
}

static bvc_status bvc_batch_project_impl(bvc_batch b, const double* coeffs, bvc_multi_cache* cache,
                                        bvc_stream stream) {
  if (coeffs == nullptr || !valid_batch_cache(b, cache)) return BVC_ERR_INVALID_ARG;
  return launch_project(coeffs, cache, (cudaStream_t)stream, b->sample_mesh, b->table);
}
extern "C" bvc_status bvc_batch_project(bvc_batch b, const double* coeffs, bvc_multi_cache* cache,
                                        bvc_stream stream) {
  return bvc::note_status(bvc_batch_project_impl(b, coeffs, cache, stream));
}

// ---------------------------------------------------------------------------
// wos_estimate_static_scratch: the pointwise estimator for callers that may
// not allocate device memory.  Its scratch (walk records and the work
// counter) is this file-scope array, so it needs no workspace from the
// caller and performs no allocation.  Every GPU that loads the library keeps
// the array resident until the process exits.
namespace {
constexpr size_t kStaticScratchBytes = size_t(16) << 20;  // 16 MiB
static __device__ __align__(256) unsigned char g_wos_scratch[kStaticScratchBytes];
std::mutex g_scratch_mu;
void* g_scratch_addr[64] = {};

// Device address of the array on the current device, looked up once per
// device (host code cannot use the symbol itself as a device pointer).
bvc_status static_scratch_address(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return BVC_ERR_CUDA;
  }
  if (dev < 0 || dev >= 64) return BVC_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (g_scratch_addr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_wos_scratch) != cudaSuccess || p == nullptr) {
      (void)cudaGetLastError();
      return BVC_ERR_CUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return BVC_OK;
}
}  // namespace

static bvc_status wos_estimate_static_scratch_impl(bvc_geometry g, const bvc_function* gfn, const bvc_function* ffn,
                                                  bvc_eval_state* state, int32_t walks, float eps,
                                                  int32_t max_steps, uint64_t seed, uint64_t id_base,
                                                  bvc_stream stream) {
  if (g == nullptr || state == nullptr || walks < 1) return BVC_ERR_INVALID_ARG;
  // one point's first hit and walk records must fit beside the counter
  size_t need = 0;
  if (wos_estimate_workspace_size(g->dim, 1, walks, &need, nullptr) != BVC_OK) return BVC_ERR_INVALID_ARG;
  if (need > kStaticScratchBytes) return BVC_ERR_WORKSPACE;
  void* scratch = nullptr;
  const bvc_status st = static_scratch_address(&scratch);
  if (st != BVC_OK) return st;
  return wos_estimate(g, gfn, ffn, state, walks, eps, max_steps, seed, id_base, scratch, kStaticScratchBytes, stream);
}
extern "C" bvc_status wos_estimate_static_scratch(bvc_geometry g, const bvc_function* gfn, const bvc_function* ffn,
                                                  bvc_eval_state* state, int32_t walks, float eps,
                                                  int32_t max_steps, uint64_t seed, uint64_t id_base,
                                                  bvc_stream stream) {
  return bvc::note_status(wos_estimate_static_scratch_impl(g, gfn, ffn, state, walks, eps, max_steps, seed, id_base, stream));
}
