/*
 * bvc.h -- C ABI of the GB300 (sm_103a) Boundary Value Caching library.
 *
 * Method: Miller, Sawhney, Crane, Gkioulekas, "Boundary Value Caching for
 * Walk on Spheres", ACM TOG 42(4), SIGGRAPH 2023.  The library solves
 *     Laplacian(u) = f in Omega,  u = g on the boundary      (Eq. 1, sigma = 0,
 *                                                            Dirichlet only)
 * by the paper's cache (Alg. 1): walk on spheres (Sec. 3.1) estimates u and
 * du/dn at samples of an inward-offset boundary (Sec. 3.2); the boundary
 * integral equation (Eq. 2) is then evaluated at interior points by the
 * Monte Carlo sums of Eq. 3-6.
 *
 * Conventions for every entry point:
 *  - Plain pointers and sizes only.  "device" pointers are CUDA device
 *    memory owned by the caller (the library never frees them); "host"
 *    pointers are read during the call only.
 *  - Point arrays are structure-of-arrays: a [dim][count] float array,
 *    coordinate a of point i at index a*count + i.
 *  - Work is enqueued asynchronously on `stream` (a cudaStream_t; NULL means
 *    the legacy default stream).  Argument errors are returned synchronously
 *    and enqueue nothing.  Errors raised inside kernels (a wait that ran out,
 *    walks stopped at max_steps) are latched in the geometry's device status
 *    word; read it with bvc_geometry_stats.
 *  - Randomness is Philox-4x32-10 (Salmon et al., SC'11) keyed by the 64-bit
 *    seed, counter = (id low, id high, word2, tag); tags: 0 cache walks,
 *    1 boundary samples, 2 source samples, 3 pointwise walks.  Results are
 *    bit-reproducible for a given seed and launch-independent.
 *  - The functions g and f are sums of closed-form terms (bvc_function);
 *    they stand in for the paper's callbacks (Sec. 4 "Setup").
 *  - Nothing here allocates device memory except bvc_geometry_create,
 *    bvc_batch_create and bvc_mixed_create, which own their trees until
 *    bvc_geometry_destroy / bvc_batch_destroy / bvc_mixed_destroy; a failed
 *    allocation returns BVC_ERR_OOM and leaves *out NULL.  Scratch memory is passed in as a workspace; each
 *    *_workspace_size call says how much is needed.
 */
#ifndef BVC_H_
#define BVC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* bvc_stream;

typedef enum {
  BVC_OK = 0,
  BVC_ERR_INVALID_ARG = 1,     /* null pointer, bad size or dimension */
  BVC_ERR_DEGENERATE_MESH = 2, /* non-finite vertex, index out of range, zero-measure element */
  BVC_ERR_OOM = 3,             /* device allocation failed (geometry only) */
  BVC_ERR_CUDA = 4,            /* a CUDA runtime call failed */
  BVC_ERR_TIMEOUT = 5,         /* a bounded in-kernel wait ran out (device status) */
  BVC_ERR_UNSUPPORTED = 6,     /* valid request the library does not implement */
  BVC_ERR_WORKSPACE = 7,       /* workspace too small for even one chunk */
  BVC_WARN_WALK_CAP = 8,       /* some walks stopped at max_steps (device status) */
  BVC_ERR_BOUNDS = 9           /* a debug build's device bounds check failed (device status) */
} bvc_status;

/* ------------------------------------------------------------------ g, f */
/* A problem function (g or f of Eq. 1) is a sum of up to BVC_MAX_TERMS
 * closed-form terms; coefficients are read on the host during the call.
 *   BVC_FN_POLY: monomials x^i y^j (z^k) of total degree <= 4, ordered by
 *     degree t = 0..4, then i = t..0, then (3D) j = t-i..0; up to 15 (2D) or
 *     35 (3D) coefficients, missing trailing ones are zero.
 *   BVC_FN_GAUSS: [s, A_1, c_1 (dim), A_2, c_2, ...] ->
 *     sum_k A_k exp(-|x - c_k|^2 / (2 s^2)).
 *   BVC_FN_GAUSS_LAPLACIAN: same coefficients -> the Laplacian of GAUSS,
 *     sum_k A_k (|x - c_k|^2 / s^4 - dim / s^2) exp(-|x - c_k|^2 / (2 s^2)).
 *   BVC_FN_EXP_TRIG (3D): [A, alpha, beta, gamma] ->
 *     A exp(alpha z) cos(beta x) sin(gamma y).
 *   BVC_FN_EXP_COS: [A, alpha, beta] -> A exp(alpha x_last) cos(beta x_0)
 *     (x_last = y in 2D, z in 3D): a solution of Delta u = sigma u with
 *     sigma = alpha^2 - beta^2.
 * The total coefficient count over all terms is at most BVC_MAX_COEFFS. */
#define BVC_MAX_TERMS 4
#define BVC_MAX_COEFFS 120
typedef enum {
  BVC_FN_POLY = 1,
  BVC_FN_GAUSS = 2,
  BVC_FN_GAUSS_LAPLACIAN = 3,
  BVC_FN_EXP_TRIG = 4,
  BVC_FN_EXP_COS = 5
} bvc_fn_kind;
typedef struct {
  int32_t kind;
  int32_t n_coeffs;
  const double* coeffs; /* host */
} bvc_term;
typedef struct {
  int32_t n_terms; /* 0 = the zero function */
  bvc_term terms[BVC_MAX_TERMS];
} bvc_function;

/* -------------------------------------------------------------- geometry */
/* Boundary mesh and its closest-point BVH (Sec. 4 "Setup": a bounding
 * volume hierarchy answers the closest-point queries of walk on spheres).
 * dim = 2: counter-clockwise polygon(s), prims = segment vertex pairs.
 * dim = 3: triangles wound counter-clockwise seen from outside.
 * verts: host float[n_verts][dim] (row-major); prims: host int32[n_prims][dim].
 * Validation: finite vertices, indices in range, no zero-length or
 * zero-area element (BVC_ERR_DEGENERATE_MESH).  The BVH is built on the host
 * (binned SAH) and copied to device memory the handle owns.  The allocation
 * is stream-ordered (cudaMallocAsync on `stream`) and the copies are
 * enqueued on `stream`, so the handle is ready for later work on that
 * stream at once (other streams must first synchronise with it); the call
 * does not wait for the device, and the caller's arrays are read during the
 * call only.  bvc_geometry_destroy frees with cudaFree (which waits).  The
 * handle also holds the element-measure CDF used by boundary sampling
 * (Sec. 4 "Sampling"), the per-vertex displacements of the offset boundary
 * (Sec. 3.2, see bvc_sample_boundary) and a small device status/statistics
 * block. */
typedef struct bvc_geometry_s* bvc_geometry;

bvc_status bvc_geometry_create(int32_t dim, const float* verts, int64_t n_verts, const int32_t* prims,
                               int64_t n_prims, bvc_stream stream, bvc_geometry* out);
bvc_status bvc_geometry_destroy(bvc_geometry g);

typedef struct {
  int32_t dim;
  int64_t n_verts, n_prims, n_nodes;
  double boundary_measure; /* |dOmega|: total length (2D) or area (3D), FP64 sequential sum */
  float bbox_lo[3], bbox_hi[3];
  size_t device_bytes; /* device memory owned by the handle */
  double offset_reach; /* max_v |m_v| >= 1: the offset boundary at l lies within l x reach of the boundary */
} bvc_geometry_info;
bvc_status bvc_geometry_get_info(bvc_geometry g, bvc_geometry_info* info);

/* Device status/statistics block: out[0] total walk steps (closest-point
 * queries made by walks), out[1] walks stopped at max_steps, out[2] error
 * flags (bit 0: timeout, bit 1: a bounds check of a debug build failed),
 * out[3] internal, out[4] BVH nodes fetched and
 * out[5] primitives tested by walks while counting is on, out[6..7]
 * reserved.  Synchronises `stream`.  With reset != 0 the block is cleared
 * after reading.  Returns BVC_ERR_BOUNDS if bit 1 is set, else
 * BVC_ERR_TIMEOUT if bit 0 is, else BVC_WARN_WALK_CAP if capped walks were
 * seen. */
bvc_status bvc_geometry_stats(bvc_geometry g, uint64_t out[8], int32_t reset, bvc_stream stream);

/* Counting mode (on != 0): later walks on this geometry run a variant that
 * also counts BVH node fetches and primitive tests into the status block,
 * from which the algorithmic bytes of a walk step are derived.  The walks'
 * results are identical in both modes; counting costs a little speed. */
bvc_status bvc_geometry_set_counting(bvc_geometry g, int32_t on);

/* Closest boundary point of m query points (the query WoS makes each step,
 * Sec. 3.1).  pts: device [dim][m].  d2: device float[m], squared distance;
 * prim: device int32[m], index of the closest element in the caller's
 * numbering (ties -> lowest index); cp: device float[dim][m] closest points
 * or NULL.  The distance is the canonical FP32 expression documented in
 * csrc/bvc_device.cuh, so the chosen index is reproducible bit for bit. */
bvc_status bvc_query_closest(bvc_geometry g, const float* pts, int64_t m, float* d2, int32_t* prim, float* cp,
                             bvc_stream stream);

/* Flag evaluation points that may lie outside the region bounded by the
 * offset boundary at `l` (Sec. 3.2: such points get pointwise walk-on-
 * spheres estimates instead of the cache): near: device uint8[m], 1 if the
 * distance to the boundary is below l x offset_reach (bvc_geometry_info;
 * every point of the strip between the boundary and the offset boundary is
 * that close). */
bvc_status bvc_classify_near(bvc_geometry g, const float* pts, int64_t m, float l, uint8_t* near,
                             bvc_stream stream);

/* ----------------------------------------------------- cache build steps */
/* K1 -- boundary samples (Alg. 1 "b.z, b.n_z ~ p", Sec. 4 "Sampling",
 * Sec. 3.2 offset boundary).  The offset boundary at l is the closed
 * surface of the mesh with every vertex v moved to v - l m_v, the region it
 * bounds being the one the cache's integral equation (Eq. 2) and source
 * samples refer to: in 2D m_v is the miter of the vertex's two segments
 * with normals na, nb, (na + nb) / max(1 + na.nb, 1/4), so each moved
 * segment is parallel to its element at distance l (any other number k of
 * segments: their normals' sum, normalised); in 3D m_v = N^ / max(min_f
 * n_f . N^, 1/4) with N^ the angle-weighted vertex normal, so no incident
 * face moves by less than l.  Sample i draws Philox(id = i, word2 = 0,
 * tag = 1) -> (u0, u1, u2); s = (i + u0)/n selects the element by the FP64
 * CDF of element measures (stratified); in 2D the remainder of s inside the
 * element is the arclength fraction, in 3D (u1, u2) give the barycentrics
 * 1 - sqrt(u1), sqrt(u1)(1 - u2), sqrt(u1) u2.  The sample is the point with
 * those coordinates on the MOVED element (FP64, rounded to FP32), nrm the
 * moved element's outward unit normal, and jac = |moved element| /
 * |element|, so that 1/p = |dOmega| jac.  l = 0 gives points on the mesh
 * and jac = 1.  z, nrm: device float[dim][n]; jac: device float[n];
 * elem: device int32[n] or NULL. */
bvc_status bvc_sample_boundary(bvc_geometry g, int64_t n, double l, uint64_t seed, float* z, float* nrm, float* jac,
                               int32_t* elem, bvc_stream stream);

/* K2 / K6 -- walks on spheres (Sec. 3.1) from n start points, `walks` each;
 * walk j of start i has id = id_base + i*walks + j and step k draws
 * Philox(id, word2 = k, tag).  Each step: closest point (distance R); stop
 * if R < eps (return g at the closest point) or after max_steps queries;
 * else direction w uniform on the sphere, source point y = x + R u2 w with
 * weights w_u = -R rho ln(R/rho) (2D) or -rho(R - rho) (3D) on f(y) (ball
 * Green's function), and x += R w.  The first step also gives the gradient
 * estimate of Eq. 7 with control variate g(closest point of the start):
 *   grad = w0 [ (dim/R0)(U - w_u,0 f(y0) - g(pbar0)) - R0 (1 - (rho0/R0)^dim) f(y0) ].
 * Output per walk t (t = i*walks + j), FP32, structure of arrays:
 *   rec[t]                    U (estimate of u at the start)
 *   rec[n*walks*(1+a) + t]    if nrm != NULL: a = 0 only, n_i . grad (du/dn);
 *                             else a = 0..dim-1, grad component a.
 * starts, nrm: device float[dim][n]; rec: device float[(1 + planes) * n * walks]
 * with planes = 1 (nrm given) or dim.  steps, prim: device int32[n*walks] or
 * NULL (per-walk step count and last closest element, for replay checks).
 * Step totals and capped-walk counts go to the geometry's status block,
 * whose spare word also serves as this call's work counter: bvc_walk calls
 * on one geometry must not overlap on the GPU (the chunked drivers below
 * keep their counter in their workspace instead). */
bvc_status bvc_walk(bvc_geometry g, const bvc_function* gfn, const bvc_function* ffn, const float* starts,
                    const float* nrm, int64_t n, int32_t walks, float eps, int32_t max_steps, uint64_t seed,
                    uint64_t id_base, uint32_t tag, float* rec, int32_t* steps, int32_t* prim, bvc_stream stream);

/* K3 -- per-start reduction of walk records (Alg. 1: the pointwise
 * estimates of a boundary sample).  rec as written by bvc_walk with
 * `planes` extra planes.  mode 0: out[p][i] = mean_j rec[p][i*walks + j];
 * mode 1: out[p][i] += sum_j rec[p][i*walks + j] (progressive sums).
 * out: device double[(1 + planes)][n].  Deterministic fixed-order FP64 sums. */
bvc_status bvc_reduce_walks(const float* rec, int64_t n, int32_t walks, int32_t planes, int32_t mode, double* out,
                            bvc_stream stream);

/* The boundary and source caches (Alg. 1 boundarySamples / sourceSamples).
 * All arrays are caller-owned device memory of the stated sizes. */
typedef struct {
  int32_t dim;
  int64_t n;            /* N boundary samples */
  float* z;             /* [dim][n] sample positions on the offset boundary */
  float* nrm;           /* [dim][n] unit outward normals */
  float* jac;           /* [n] measure ratios of the samples' offset elements (1/p = bnd_measure jac) */
  double* u_hat;        /* [n] estimates of u */
  double* dudn_hat;     /* [n] estimates of du/dn */
  float* packed;        /* [n][20] gather tiles, written by bvc_cache_pack */
  double bnd_measure;   /* |dOmega| = 1/p of the boundary samples */
  int64_t n_src_cand;   /* source candidates M (denominator of Eq. 4/6); 0 = no source cache */
  float* src_y;         /* [dim][n_src_cand] kept source points (first n_src_dev[0] valid) */
  double* src_c;        /* [n_src_cand] f(y) / p for kept points */
  float* src_packed;    /* [n_src_cand][8] gather tiles */
  int64_t* n_src_dev;   /* [1] number of kept source samples (written on device) */
  double sigma;         /* screening coefficient of the cache (set by the build); 0 = Poisson */
  double clamp_c;       /* bound c of the clamped dG/dn in the u term (Sec. 3.3, set by the build); 0 = none */
} bvc_cache;

/* K4 -- source samples (Alg. 1 "y ~ p^R", Sec. 4 "Sampling"): a jittered
 * grid[0] x grid[1] (x grid[2] in 3D) grid of candidates over the
 * boundary's bounding box; candidate c (cell c mod G0, (c / G0) mod G1,
 * c / (G0 G1)) draws Philox(id = c, word2 = 0, tag = 2) for its position in
 * its cell.  The region is the one inside the offset boundary at offset_l
 * (Sec. 3.2; its vertices fl32(v - offset_l m_v), see bvc_sample_boundary;
 * 0 = the mesh itself).  2D: kept when the canonical FP32 crossing test puts
 * it inside that polygon.  3D: kept when the generalized winding number of that mesh
 * (the sum of its triangles' signed solid angles over 4 pi, FP32) is above
 * 1/2 -- 1 inside a closed outward-wound surface, so holes are wound
 * inward; overlapping shells are counted with their orientation, not
 * repaired.  With p = 1/|box| on the box times the indicator of Omega, a
 * kept sample carries c = f(y) |box| and the estimator divides by the
 * candidate count.  Kept samples are stored in candidate order.  Requires
 * cache->n_src_cand = the grid's cell count.  Workspace:
 * bvc_sample_source_workspace_size. */
bvc_status bvc_sample_source_workspace_size(int64_t n_cand, size_t* bytes);
bvc_status bvc_sample_source(bvc_geometry g, const bvc_function* ffn, const int32_t grid[3], uint64_t seed,
                             double offset_l, bvc_cache* cache, void* workspace, size_t workspace_bytes,
                             bvc_stream stream);

/* Pack z, nrm, u_hat, dudn_hat (and the kept source samples) into the
 * gather's tile layout, folding 1/p = bnd_measure jac and the Green's
 * function constants of App. A into the per-sample coefficients. */
bvc_status bvc_cache_pack(const bvc_cache* cache, bvc_stream stream);

typedef struct {
  int64_t n_samples;        /* N */
  int32_t walks_per_sample; /* nWalks of Alg. 1 */
  int32_t max_steps;        /* cap on closest-point queries per walk (e.g. 1 << 14) */
  double offset_l;          /* Sec. 3.2 offset l > eps of the offset boundary (see bvc_sample_boundary) */
  double eps;               /* epsilon shell width */
  uint64_t seed;
  uint64_t walk_id_base;    /* first walk id: distinct caches of one seed use disjoint ranges */
  int32_t src_grid[3];      /* source candidate grid (2D: [0] x [1], [2] unused; 3D: all three),
                               all 0 = no source cache */
  double sigma;             /* screened Poisson (Delta - sigma) u = f when > 0 (Eq. 1): the walks
                               weight each ball by its screened mean-value factor and each step's
                               source sample by the screened ball Green's function (see
                               wos_estimate_sigma); the gather uses the screened Green's functions
                               of App. A for the boundary and the source samples.  0 = Poisson. */
  double clamp_c;           /* > 0: the gather clamps dG/dn in the u term to [-c, c] (Sec. 3.3,
                               Eq. 8-9); bvc_clamp_correction estimates the remainder.  0 = none. */
  int32_t reuse_sources;    /* != 0: cache->src_y and n_src_dev already hold the kept source
                               candidates of this geometry, grid and seed (an earlier build); only
                               their weights f(y) |box| are recomputed -- the same values a full
                               build gives, without the inside tests. */
} bvc_cache_opts;

/* The whole cache: K1 -> K2 (chunked through the workspace) -> K3 -> K4 (in
 * the region inside the offset boundary at opts->offset_l) -> pack.
 * cache->n must equal opts->n_samples; n_src_cand must equal the grid size.
 * Any workspace of at least bvc_cache_build_workspace_size(min) bytes works;
 * larger ones (up to `full`) run the walks in fewer chunks. */
bvc_status bvc_cache_build_workspace_size(bvc_geometry g, const bvc_cache_opts* opts, size_t* min_bytes,
                                          size_t* full_bytes);
bvc_status bvc_cache_build(bvc_geometry g, const bvc_function* gfn, const bvc_function* ffn,
                           const bvc_cache_opts* opts, bvc_cache* cache, void* workspace, size_t workspace_bytes,
                           bvc_stream stream);

/* ------------------------------------------------------------ evaluation */
/* Running sums of Alg. 1's EvaluationPoint for m points (every point of a
 * set receives the same samples, so the counts are kept once per set). */
typedef struct {
  int32_t dim;
  int64_t m;
  const float* x;   /* [dim][m] evaluation points */
  double* u_bnd;    /* [m] sum of boundary terms (Eq. 3 numerators) */
  double* u_src;    /* [m] sum of source terms (Eq. 4) */
  double* grad_bnd; /* [dim][m] Eq. 5 sums, or NULL */
  double* grad_src; /* [dim][m] Eq. 6 sums, or NULL */
  int64_t* counts;  /* [2] N and M accumulated so far */
} bvc_eval_state;

/* K5 -- the all-pairs gather (Alg. 1 splat loops, Eq. 3-6): adds every
 * cache sample's contribution to every point's sums and adds N and M to the
 * counts.  Cache tiles are staged in shared memory by bulk asynchronous
 * copies (TMA); pair terms are FP32, partial sums over at most 128 samples
 * are flushed to FP64.  Workspace: bvc_evaluate_workspace_size. */
bvc_status bvc_evaluate_workspace_size(const bvc_cache* cache, const bvc_eval_state* state, size_t* bytes);
bvc_status bvc_evaluate(const bvc_cache* cache, bvc_eval_state* state, void* workspace, size_t workspace_bytes,
                        bvc_stream stream);

/* Gather autotuner (the gather's analogue of bvc_tune_walks): the gathers
 * give each thread several evaluation points, every sample staged in shared
 * memory serving all of them; more points per thread mean fewer shared
 * loads per pair but more registers.  bvc_tune_gather times two launches of
 * each supported count (2, 4, 6 for boundary samples, 2, 4 for sources) of
 * this cache's gathers at the points of `state` (CUDA events on `stream`;
 * synchronous, so not for stream capture), keeps the fastest for all later
 * gathers of that dimension and kind in this process, returns them in
 * pts_out = {boundary, source} and their summed time in best_ms (may be
 * NULL), and clears the state's sums.  A screened or clamped cache's
 * boundary gather (a separate kernel) is not tuned.  Workspace as
 * bvc_evaluate (bvc_evaluate_workspace_size covers every count).
 * bvc_set_gather_shape sets a count by hand (kind 0 boundary, 1 source;
 * pts 0 = the built-in default).  Results do not depend on the counts. */
bvc_status bvc_tune_gather(const bvc_cache* cache, bvc_eval_state* state, void* workspace, size_t workspace_bytes,
                           bvc_stream stream, int32_t pts_out[2], float* best_ms);
bvc_status bvc_set_gather_shape(int32_t dim, int32_t kind, int32_t pts);

/* Zero the running sums and counts of a state (cudaMemsetAsync, no kernel). */
bvc_status bvc_eval_state_reset(const bvc_eval_state* state, bvc_stream stream);

/* a6 -- Alg. 1 GetSolution: u = u_bnd/N + u_src/M (a term is dropped when
 * its count is 0); grad likewise.  u: device double[m]; grad: device
 * double[dim][m] or NULL. */
bvc_status bvc_get_solution(const bvc_eval_state* state, double* u, double* grad, bvc_stream stream);

/* K6 -- pointwise walk on spheres at the m points of `state` (the
 * comparison estimator, and the estimate used within l of the boundary,
 * Sec. 3.2): `walks` walks per point with tag 3, ids id_base + k*walks + j.
 * The walks' sums go into the state's running sums like a cache's would:
 * u_bnd[k] += sum_j U, grad_bnd[a][k] += sum_j grad_a (if grad_bnd is set),
 * counts[0] += walks -- so bvc_get_solution returns the pointwise means and
 * successive calls with disjoint id ranges refine them progressively.
 * Workspace chunks the walks by points. */
bvc_status wos_estimate_workspace_size(int32_t dim, int64_t m, int32_t walks, size_t* min_bytes,
                                       size_t* full_bytes);
bvc_status wos_estimate(bvc_geometry g, const bvc_function* gfn, const bvc_function* ffn, bvc_eval_state* state,
                        int32_t walks, float eps, int32_t max_steps, uint64_t seed, uint64_t id_base,
                        void* workspace, size_t workspace_bytes, bvc_stream stream);

/* Gather device status word (bit 0: a bounded wait for a tile copy ran
 * out; bit 1: the self-test's wait ran out).  Synchronises the device;
 * reset != 0 clears it. */
bvc_status bvc_gather_status(uint64_t* flags, int32_t reset);
/* Failure-path self-test: one warp waits on a barrier that nothing completes,
 * with the gathers' bounded wait cut to limit_ns (0..2e9); the wait gives up,
 * sets bit 1 of the status word and the kernel returns (the context stays
 * usable). */
bvc_status bvc_wait_selftest(int64_t limit_ns, bvc_stream stream);

/* ------------------------------------------------------- walk autotuner */
/* The walk kernel is persistent: a grid of (blocks per SM) x (SMs) blocks
 * pulls walks from a counter, a warp taking `chunk` walks at a time.  A
 * walk's result depends only on its id, so the shape changes speed, never
 * results.  bvc_tune_walks times the cache walks of min(N, 16384) boundary
 * samples of the given problem for every shape with blocks per SM from the
 * kernel's maximum occupancy down to half of it and chunks of 64, 128, 256
 * (best of two launches each, CUDA events on `stream`; synchronous, so not
 * for stream capture), keeps the fastest in the geometry for all later walk
 * launches on it, and returns it in shape[2] = {blocks per SM, chunk} and
 * its time in best_ms.  The tuning walks add to the geometry's status
 * block.  bvc_geometry_set_walk_shape sets a shape by hand (0 = default). */
bvc_status bvc_tune_walks_workspace_size(bvc_geometry g, const bvc_cache_opts* opts, size_t* bytes);
bvc_status bvc_tune_walks(bvc_geometry g, const bvc_function* gfn, const bvc_function* ffn,
                          const bvc_cache_opts* opts, void* workspace, size_t workspace_bytes, bvc_stream stream,
                          int32_t shape[2], float* best_ms);
bvc_status bvc_geometry_set_walk_shape(bvc_geometry g, int32_t blocks_per_sm, int32_t chunk);

/* ------------------------------------------- regions and clamped kernels */
/* Region of interest (Sec. 3.2 "Boundary Specification"): the boundary
 * samples lie on the region's own boundary (offset_l >= 0 from it, normals
 * outward of the region), the walks run in the domain (its geometry), the
 * source samples fill the region (its bounding box and inside test), and the
 * gather then evaluates u and grad u at points inside the region (the
 * estimate is 0 outside it).  region must lie inside the domain; both share
 * a dimension.  Otherwise as bvc_cache_build. */
bvc_status bvc_cache_build_region(bvc_geometry domain, bvc_geometry region, const bvc_function* gfn,
                                  const bvc_function* ffn, const bvc_cache_opts* opts, bvc_cache* cache,
                                  void* workspace, size_t workspace_bytes, bvc_stream stream);

/* The remainder of the clamped double-layer kernel (Sec. 3.3, Eq. 8): for a
 * cache built with opts.clamp_c = c (its gather uses dG/dn clamped to
 * [-c, c] in the u term), u_corr[x] (device double[m], overwritten) is an
 * unbiased estimate of int [dG/dn - clamp_c(dG/dn)] u dz over the sample
 * surface -- the offset boundary of `surface` at offset_l (its vertices
 * moved by -offset_l m_v as in bvc_sample_boundary: the cache's geometry and
 * offset, or a region and 0) -- so that get_solution + u_corr
 * is unbiased.  n_dirs directions per point (Philox id = point * n_dirs + j,
 * word2 0, tag 4) sample the signed solid angle; every crossing closer than
 * 1/(2 pi c) (2D) or (4 pi c)^(-1/2) (3D) with |dG/dn| > c adds
 * sign(n.w) (1 - c/|dG/dn|) u(z) / n_dirs, u(z) from `walks` walks on the
 * domain (tag 5, ids rank * walks + j, crossings ranked by point, direction,
 * distance; at most 8 per ray).  Synchronises `stream` once (the crossing
 * count decides the walk launches); *n_hits receives that count. */
bvc_status bvc_clamp_correction_workspace_size(int32_t dim, int64_t m, int32_t n_dirs, int32_t walks,
                                               size_t* min_bytes);
bvc_status bvc_clamp_correction(bvc_geometry domain, bvc_geometry surface, double offset_l, const bvc_function* gfn,
                                const bvc_function* ffn, double sigma, double clamp_c, const float* pts, int64_t m,
                                int32_t n_dirs, int32_t walks, float eps, int32_t max_steps, uint64_t seed,
                                double* u_corr, int64_t* n_hits, void* workspace, size_t workspace_bytes,
                                bvc_stream stream);

/* ------------------------------------------------------ differentiation */
/* Gradients of a loss L of the values u(x) that bvc_evaluate gives (Eq. 3)
 * with respect to the boundary data and the source.  The parameters are
 *   - g as values at the mesh vertices (device float[n_verts]), interpolated
 *     linearly on the element holding a walk's closest point (segment:
 *     projection parameter; triangle: barycentric coordinates), and
 *   - the amplitudes A_k of f when f is one BVC_FN_GAUSS or
 *     BVC_FN_GAUSS_LAPLACIAN term of at most 8 bumps (f = sum_k A_k psi_k).
 * With fixed seeds the walks' paths depend on neither, and every estimate
 * (U, n.grad per walk; u^, du/dn^ per sample; the source weights c; u(x)) is
 * linear in both, so the gradient is exact for the estimator: the adjoint
 * of the gather gives dL/du^, dL/d(du/dn^) and dL/dc per sample
 * (bvc_evaluate_adjoint), and the adjoint of the cache build replays each
 * walk from its Philox stream and adds its weights to the vertices of the
 * elements where it ends and starts and to the amplitudes
 * (bvc_cache_adjoint).  Gradient sums are FP64; vertex gradients are
 * accumulated with FP64 atomics (order-dependent in the last bits). */

/* bvc_cache_build with g given by vertex values (device float[n_verts]). */
bvc_status bvc_cache_build_vg(bvc_geometry g, const float* g_vertex, const bvc_function* ffn,
                              const bvc_cache_opts* opts, bvc_cache* cache, void* workspace, size_t workspace_bytes,
                              bvc_stream stream);
bvc_status bvc_evaluate_adjoint_workspace_size(int64_t m, size_t* bytes);
/* lam: device double[m], dL/du at the points pts (device [dim][m]) of one
 * bvc_evaluate of this cache (one cache per evaluation state, so u = sums /
 * (n, n_src_cand)).  Writes adj_u, adj_q (device double[n]) and, if
 * adj_src is non-NULL and the cache has source candidates, adj_src (device
 * double[n_src_cand], zero past the kept ones).  Poisson caches only: a
 * screened or clamped cache returns BVC_ERR_UNSUPPORTED. */
bvc_status bvc_evaluate_adjoint(const bvc_cache* cache, const float* pts, int64_t m, const double* lam,
                                double* adj_u, double* adj_q, double* adj_src, void* workspace,
                                size_t workspace_bytes, bvc_stream stream);
bvc_status bvc_cache_adjoint_workspace_size(bvc_geometry g, const bvc_cache_opts* opts, size_t* min_bytes,
                                            size_t* full_bytes);
/* Adds dL/dg_vertex into grad_gv (device double[n_verts]) and dL/dA into
 * grad_amp (device double[8], used when f has a term) for the cache built by
 * bvc_cache_build_vg with the same geometry, f, opts (seed, ids) -- its
 * samples z, n are read from `cache`.  adj_src may be NULL (no source
 * cache).  BVC_ERR_UNSUPPORTED if f is not of the differentiable form. */
bvc_status bvc_cache_adjoint(bvc_geometry g, const bvc_function* ffn, const bvc_cache_opts* opts,
                             const bvc_cache* cache, const double* adj_u, const double* adj_q, const double* adj_src,
                             double* grad_gv, double* grad_amp, void* workspace, size_t workspace_bytes,
                             bvc_stream stream);

/* ---------------------------------------------- many right-hand sides */
/* Batching of right-hand sides: K Dirichlet data g_k = sum_m C[k][m] phi_m
 * over the BVC_FN_POLY monomials phi_m (total degree <= 4;
 * bvc_poly_terms(dim) = 15 in 2D, 35 in 3D), and, with
 * bvc_multi_cache_build_source, K sources f_k = sum_b A[k][b] psi_b over the
 * bumps psi_b of one shared GAUSS or GAUSS_LAPLACIAN term.
 * Without a source term a walk's path does not depend on g and each walk's
 * U and n.grad (Sec. 3.1, Eq. 7) are linear in g, so one set of walks per
 * cache serves every right-hand side: the walks record their end points,
 * per-sample moments of the monomials are reduced once (FP64), and each
 * right-hand side's u^ and du/dn^ are projections of the moments -- the
 * estimates the single-RHS path gives for g_k, up to rounding.  The gather
 * then evaluates Eq. 3 for all right-hand sides at once.  With a source the
 * walks' paths still do not depend on (g, f) (a step's source point is drawn
 * from the step's own ball), each walk also records, per bump, its source
 * sums; their per-sample means join the moments, and the source candidates
 * of Eq. 4 join the gather as extra rows whose per-RHS weights are
 * projections of the candidates' bump values.  All arrays are
 * caller-owned device memory. */
#define BVC_MULTI_GROUP 32 /* right-hand sides per gather pass */
typedef struct {
  int32_t dim;
  int64_t n;           /* boundary samples */
  int32_t k;           /* right-hand sides */
  float* z;            /* [dim][n] */
  float* nrm;          /* [dim][n] */
  float* jac;          /* [n] measure ratios (1/p = |dOmega| jac) */
  double* mom_u;       /* [n][bvc_poly_terms(dim)] means of phi_m at walk ends */
  double* mom_q;       /* [n][bvc_poly_terms(dim)] means of s (phi_m(end) - phi_m(p0)) */
  double* u_hat;       /* [k][n] */
  double* dudn_hat;    /* [k][n] */
  float* packed;       /* [ceil(k/32)][n + n_src_cand][8 + 64] gather tiles */
  double bnd_measure;  /* |dOmega|, set by the build */
  /* Source part (bvc_multi_cache_build_source; 0 / NULL for Laplace): */
  int32_t n_bumps;     /* B <= 8 bumps of the shared source term (set by the build) */
  double* mom_su;      /* [n][8] per-sample means over walks of sum_steps w_u psi_b(y) */
  double* mom_sq;      /* [n][8] per-sample means of bump b's part of the du/dn sample */
  int64_t n_src_cand;  /* M source candidates (the grid of opts->src_grid) */
  float* src_y;        /* [dim][M] kept candidates first (Eq. 4 points) */
  float* src_psi;      /* [M][8] |box| psi_b(y_j) of the kept candidates */
  int64_t* n_src_dev;  /* device int64: candidates kept */
} bvc_multi_cache;

int32_t bvc_poly_terms(int32_t dim);
bvc_status bvc_multi_cache_build_workspace_size(bvc_geometry g, int64_t n, int32_t walks, size_t* min_bytes,
                                                size_t* full_bytes);
/* K1 boundary samples, end-point walks (tag 0, ids as bvc_cache_build),
 * moments and the projection onto coeffs (device double[k][terms]).
 * opts->src_grid must be {0, 0} (BVC_ERR_UNSUPPORTED otherwise). */
bvc_status bvc_multi_cache_build(bvc_geometry g, const double* coeffs, const bvc_cache_opts* opts,
                                 bvc_multi_cache* cache, void* workspace, size_t workspace_bytes, bvc_stream stream);
/* The same with a source term: f_k = sum_b A[k][b] psi_b, psi_b the bumps of
 * `shape` (one term of kind BVC_FN_GAUSS or BVC_FN_GAUSS_LAPLACIAN, 1..8
 * bumps; its amplitudes are not used).  coeffs: device double[k][terms + B]
 * (each row: the monomial coefficients of g_k, then A[k][0..B)).  The
 * walks, their draws and the source candidates (opts->src_grid >= 1 each,
 * cache->n_src_cand = their count; seed opts->seed; kept inside the offset
 * boundary at opts->offset_l) are those of bvc_cache_build with f_k, so each
 * right-hand side's u^, du/dn^ and Eq. 3 + Eq. 4 value equal the single-RHS
 * results up to rounding.  Workspace: bvc_multi_cache_build_source_workspace_size. */
bvc_status bvc_multi_cache_build_source_workspace_size(bvc_geometry g, const bvc_cache_opts* opts, size_t* min_bytes,
                                                       size_t* full_bytes);
bvc_status bvc_multi_cache_build_source(bvc_geometry g, const bvc_function* shape, const double* coeffs,
                                        const bvc_cache_opts* opts, bvc_multi_cache* cache, void* workspace,
                                        size_t workspace_bytes, bvc_stream stream);
/* Re-project the stored moments onto new coefficients (no walks); with a
 * source (cache->n_bumps > 0) the rows of coeffs hold terms + n_bumps values. */
bvc_status bvc_multi_cache_project(const double* coeffs, bvc_multi_cache* cache, bvc_stream stream);
/* Eq. 3 for every right-hand side at m points: u[k][x] = (1/n) sum_i
 * (dG/dn(x, z_i) u^_ik - G(x, z_i) du/dn^_ik) / p  (overwritten; u only),
 * plus Eq. 4's (1/M) sum_j G(x, y_j) c_jk over the kept candidates when the
 * cache has a source.  pts: device [dim][m]; u: device double[k][m]. */
bvc_status bvc_evaluate_multi(const bvc_multi_cache* cache, const float* pts, int64_t m, double* u,
                              bvc_stream stream);

/* ---------------------------------------------- many meshes in one launch */
/* A batch of independent Laplace problems on meshes of the same dimension
 * and uneven size, each with K polynomial right-hand sides as above.  The
 * batch concatenates the meshes' BVHs into one forest (indices rebased,
 * device memory owned by the batch), so the walks of every mesh run in one
 * persistent launch and the gather of every mesh in one launch.  Walk ids
 * and boundary samples are those of bvc_multi_cache_build on each mesh alone
 * with walk_id_base = (first sample of the mesh in the batch) x walks and the
 * same seed, so every mesh's results equal the single-mesh results bit for
 * bit.  bvc_batch_build and bvc_batch_evaluate only launch kernels and clear
 * device words on the stream (no allocation, no synchronisation), so they
 * may be captured in a CUDA graph. */
typedef struct bvc_batch_s* bvc_batch;
typedef struct {
  bvc_geometry geom; /* borrowed: must outlive the batch */
  int64_t n_samples; /* boundary samples (>= 1) */
  double offset_l;   /* inward offset of the samples (Sec. 3.2) */
  float eps;         /* epsilon-shell of this mesh's walks */
  int64_t n_points;  /* evaluation points (>= 0) */
} bvc_batch_mesh;

/* Builds the forest (stream-ordered on `stream`, as bvc_geometry_create).  All meshes must share one
 * dimension; count >= 1; walks, max_steps >= 1; k >= 1.  Samples of mesh j
 * occupy [sum_{i<j} n_samples_i, ...) of the batch's sample range and its
 * points [sum_{i<j} n_points_i, ...) of the point range. */
bvc_status bvc_batch_create(const bvc_batch_mesh* meshes, int32_t count, int32_t walks, int32_t max_steps,
                            int32_t k, bvc_stream stream, bvc_batch* out);
bvc_status bvc_batch_destroy(bvc_batch b);
/* Walk counters of the forest, as bvc_geometry_stats / _set_counting. */
bvc_status bvc_batch_set_counting(bvc_batch b, int32_t on);
bvc_status bvc_batch_stats(bvc_batch b, uint64_t out[8], int32_t reset, bvc_stream stream);
/* n_total, m_total: sums of n_samples and n_points. */
bvc_status bvc_batch_get_info(bvc_batch b, int32_t* dim, int64_t* n_total, int64_t* m_total);
bvc_status bvc_batch_build_workspace_size(bvc_batch b, size_t* min_bytes, size_t* full_bytes);
/* coeffs: device double[count][k][bvc_poly_terms(dim)]; cache: a
 * bvc_multi_cache with n = n_total and k = the batch's k (its bnd_measure
 * is left 0: each mesh's measure is held by the batch).  seed: a DEVICE
 * uint64 read by the kernels when they run, so a captured graph replays
 * with whatever seed the word holds at replay time. */
bvc_status bvc_batch_build(bvc_batch b, const double* coeffs, const uint64_t* seed, bvc_multi_cache* cache,
                           void* workspace, size_t workspace_bytes, bvc_stream stream);
/* Re-project the stored moments onto new coefficients (no walks). */
bvc_status bvc_batch_project(bvc_batch b, const double* coeffs, bvc_multi_cache* cache, bvc_stream stream);
/* Eq. 3 for every mesh and right-hand side: pts device [dim][m_total];
 * u device double[k][m_total] (overwritten), point p of mesh j gathered
 * over mesh j's samples only. */
bvc_status bvc_batch_evaluate(bvc_batch b, const bvc_multi_cache* cache, const float* pts, double* u,
                              bvc_stream stream);

/* wos_estimate for the screened equation (Delta - sigma) u = f (sigma >= 0).
 * Each ball of radius R multiplies the walk's weight by its screened
 * mean-value factor (R sqrt(sigma)) / sinh(R sqrt(sigma)) (3D) or
 * 1 / I0(R sqrt(sigma)) (2D); the first ball's gradient uses (dim / R) Qg
 * with Qg = t^3 / (3 (t cosh t - sinh t)) (3D) or t / (2 I1(t)) (2D),
 * t = R sqrt(sigma).  With a source, each step's sample y = x + rho w
 * (rho = R u, as for Poisson) adds, times the weight into the ball,
 * -|S| R rho^(d-1) G(rho) f(y) with G the Green's function of
 * (sigma - Delta) on the ball, zero on its sphere, seen from the centre:
 * [K0(k rho) - K0(kR) I0(k rho)/I0(kR)]/(2 pi) (2D), sinh(k (R - rho)) /
 * (4 pi rho sinh kR) (3D), k = sqrt(sigma); the gradient's first-step source
 * term uses the l = 1 radial mode of that Green's function instead (k [K1(k
 * rho) - K1(kR) I1(k rho)/I1(kR)]/(2 pi); [Q(rho) - Q(R) J(k rho)/J(kR)] /
 * (4 pi rho^2), Q(r) = e^(-kr)(kr + 1), J(t) = t cosh t - sinh t).  At sigma
 * -> 0 these are the Poisson weights.  sigma = 0 is wos_estimate. */
bvc_status wos_estimate_sigma(bvc_geometry g, const bvc_function* gfn, const bvc_function* ffn, double sigma,
                              bvc_eval_state* state, int32_t walks, float eps, int32_t max_steps, uint64_t seed,
                              uint64_t id_base, void* workspace, size_t workspace_bytes, bvc_stream stream);

/* wos_estimate with no caller workspace and no allocation.  The paper has
 * no counterpart: this is an interface for callers that must not allocate
 * device memory -- for example code that runs inside another framework
 * whose allocator owns all device memory, host callbacks where CUDA
 * allocation calls are not permitted, or latency-critical loops that cannot
 * afford the device-wide synchronisation of cudaMalloc/cudaFree.
 * The walk records live in a 16 MiB array of static device memory inside
 * this library (held on every GPU that loads the library until the process
 * exits); points are processed in chunks that fit it, so m is unbounded but
 * the scratch of one point (wos_estimate_workspace_size with m = 1) must
 * fit: walks > 1,398,057 (2D) or 1,048,542 (3D) returns BVC_ERR_WORKSPACE.
 * Arguments, results and state semantics are those of wos_estimate.  The first call on each device looks up the array's device
 * address (cudaGetSymbolAddress); make that first call before any stream
 * capture.  The address is kept for the lifetime of the device's context:
 * after cudaDeviceReset (or any teardown of the primary context) it is
 * stale, and this entry point must not be called again in that process.  All calls share the one array: calls that overlap on the GPU
 * (on different streams, or from several threads) race on it and must be
 * serialised by the caller.  The work counter in the array is cleared at
 * the start of every call. */
bvc_status wos_estimate_static_scratch(bvc_geometry g, const bvc_function* gfn, const bvc_function* ffn,
                                       bvc_eval_state* state, int32_t walks, float eps, int32_t max_steps,
                                       uint64_t seed, uint64_t id_base, bvc_stream stream);

/* ------------------------------------------- mixed boundaries (WoSt) */
/* Laplace(u) = f with u = g on the Dirichlet part and du/dn = h on the
 * Neumann part of the boundary (Eq. 1, sigma = 0), by walk on stars
 * (Sec. 3.1, Fig. "WoS vs WoSt") and the cache of Sec. 3.2 / Fig.
 * "Dirichlet offset boundary": samples on Neumann elements lie on the
 * boundary and carry the known du/dn = h(z); samples on Dirichlet elements
 * lie on the offset boundary built from the Dirichlet elements alone (as
 * bvc_sample_boundary, with displacements from the Dirichlet elements at
 * each vertex, so a vertex shared with a Neumann element moves along its
 * Dirichlet element's normal) and carry walk estimates of u and du/dn; u on
 * the Neumann samples is estimated by walks that start on the boundary.
 *
 * A walk step at x: distance d_D to the Dirichlet part (stop when below eps,
 * returning g at the closest Dirichlet point); star radius
 * R = max(min(d_D, d_sil), eps) with d_sil the distance to the closest
 * silhouette point of the Neumann part as seen from x (so each ray from x
 * crosses the Neumann part at most once inside B(x, R)); a direction w
 * uniform on the sphere (flipped into the domain when x is on the Neumann
 * part); the first crossing of x + t w, 0 < t <= R, with the Neumann part is
 * the next point (then on the boundary), else x + R w.  With r = min(t, R)
 * and rho = r u2 the step adds
 *   source  w_u f(x + rho w),  w_u = r rho ln(rho/R) (2D), -r rho (1 - rho/R) (3D)
 *   Neumann w_h h(z) at a crossing z with normal n_z,
 *           w_h = t ln(R/t)/|n_z.w| (2D), t (1 - t/R)/|n_z.w| (3D).
 * A walk that starts inside the domain first takes a ball step of radius
 * d_all (distance to the whole boundary) and estimates the gradient as
 * bvc_walk does; if d_all < eps its first step is a star step and its
 * gradient is 0.  Silhouettes: a Neumann vertex (2D) or edge (3D) between
 * two Neumann elements with outward normals n0, n1 is one when, with
 * a = (vertex or edge start) - x and d_k = n_k . a (zero when
 * |d_k| <= 2^-18 x bounding-box diagonal), one d_k is zero and the other
 * negative, or both are non-zero with opposite signs; one with one or more than two Neumann
 * elements (and no Dirichlet element) always is; one touching a Dirichlet
 * element is skipped (d_D covers it).  Draws: Philox(walk id, step - 1, tag)
 * as bvc_walk. */
typedef struct bvc_mixed_s* bvc_mixed;

/* Flags neumann[e] != 0 mark Neumann elements (host uint8[n_prims]); at
 * least one element must be Dirichlet.  Builds the whole boundary's geometry,
 * the Dirichlet and Neumann parts' geometries and the silhouette tree
 * (stream-ordered on `stream`, as bvc_geometry_create).  Mesh arguments as bvc_geometry_create. */
bvc_status bvc_mixed_create(int32_t dim, const float* verts, int64_t n_verts, const int32_t* prims, int64_t n_prims,
                            const uint8_t* neumann, bvc_stream stream, bvc_mixed* out);
bvc_status bvc_mixed_destroy(bvc_mixed m);
typedef struct {
  int32_t dim;
  int64_t n_dirichlet, n_neumann; /* elements */
  int64_t n_silhouette;           /* silhouette candidates (vertices 2D, edges 3D) */
  int64_t n_silhouette_tree;      /* those in the silhouette tree: all but the flat ones (two elements
                                     with equal normals, which are never silhouettes) */
  double dirichlet_measure, neumann_measure;
  size_t device_bytes;            /* the silhouette tree and maps (geometries not included) */
} bvc_mixed_info;
bvc_status bvc_mixed_get_info(bvc_mixed m, bvc_mixed_info* info);
/* Star radius of the walks on stars (Sec. 3.1): every step uses a ball of
 * radius R with R <= min(d_Dirichlet, d_silhouette), which keeps the ball
 * free of Dirichlet points and star-shaped about its centre, so any such R
 * gives the same (unbiased) estimator.  gap = 0 (the default) takes the
 * closest silhouette point exactly; 0 < gap < 1 lets the silhouette search
 * stop early and use a certified lower bound r of the silhouette distance
 * with (1 - gap) d_silhouette <= r <= d_silhouette (the search skips tree
 * nodes not nearer than (1 - gap) x the best so far and keeps the least
 * skipped distance).  Applies to every later call on m (walks, caches and
 * bvc_mixed_query).  Host only; gap outside [0, 1): BVC_ERR_INVALID_ARG. */
bvc_status bvc_mixed_set_silhouette_gap(bvc_mixed m, double gap);
/* Borrowed handles (owned by m): the whole boundary, its Dirichlet part and
 * its Neumann part (NULL when there is no Neumann element).  Element ids of
 * the parts are their positions among the whole mesh's Dirichlet / Neumann
 * elements. */
bvc_status bvc_mixed_geometries(bvc_mixed m, bvc_geometry* whole, bvc_geometry* dirichlet, bvc_geometry* neumann);

/* Neumann data h(z) = value(z) + n_z . grad potential(z) (either may have
 * no terms; potential kinds POLY, GAUSS, GAUSS_LAPLACIAN, EXP_TRIG, EXP_COS). */
typedef struct {
  bvc_function value;
  bvc_function potential;
} bvc_neumann;

/* Queries behind the walk, for checks: per point (device [dim][m]) the
 * distance to the Dirichlet part and to the closest silhouette point (FP32,
 * +inf when there is none); per ray (origins and unit directions device
 * [dim][m], skip: device int32[m] Neumann element to ignore, or NULL) the
 * first crossing t with the Neumann part in (0, tmax] and its Neumann element
 * id (-1 and +inf when none). */
bvc_status bvc_mixed_query(bvc_mixed m, const float* pts, int64_t n, float* d_dir, float* d_sil, bvc_stream stream);
bvc_status bvc_mixed_rays(bvc_mixed m, const float* org, const float* dir, const int32_t* skip, int64_t n,
                          float tmax, float* t, int32_t* elem, bvc_stream stream);

/* Walks on stars from n starts (device float[dim][n]); start_elem: device
 * int32[n], the whole-mesh element a start lies on (a Neumann element: the
 * walk starts on the boundary with normal nrm), or -1 / NULL for starts
 * inside.  Records as bvc_walk: with nrm != NULL one extra plane holding
 * n . grad for starts inside and h(start) for starts on the Neumann part;
 * else dim planes of grad.  steps, prim: per-walk step count and the whole-
 * mesh Dirichlet element of the end, or NULL.  Walk ids id_base + i*walks + j;
 * `counter`: device uint64 work counter, zeroed by the call. */
bvc_status bvc_mixed_walk(bvc_mixed m, const bvc_function* gfn, const bvc_neumann* h, const bvc_function* ffn,
                          const float* starts, const int32_t* start_elem, const float* nrm, int64_t n, int32_t walks,
                          float eps, int32_t max_steps, uint64_t seed, uint64_t id_base, uint32_t tag, float* rec,
                          int32_t* steps, int32_t* prim, unsigned long long* counter, bvc_stream stream);

/* Walks on stars for the screened equation (Delta - sigma) u = f with u = g
 * on the Dirichlet part and du/dn = h on the Neumann part (Eq. 1 with
 * sigma > 0; Sec. 3.1's walk on stars with the screened Green's functions
 * of App. A).  Arguments, records and draws as bvc_mixed_walk; sigma = 0 is
 * bvc_mixed_walk, negative or non-finite sigma BVC_ERR_INVALID_ARG.  With
 * k = sqrt(sigma) and G(rho) the Green's function of (sigma - Delta) on the
 * step's ball B(x, R) that vanishes on its sphere,
 *   2D  G = [K0(k rho) - K0(kR) I0(k rho)/I0(kR)] / (2 pi)
 *   3D  G = sinh(k (R - rho)) / (4 pi rho sinh kR),
 * every estimate the walk carries past a step is multiplied by that step's
 * factor: the gradient ball's mean-value factor C (t / sinh t in 3D,
 * 1 / I0(t) in 2D, t = kR), and for a star step whose direction meets the
 * boundary first at distance r (r = R when it meets the sphere)
 * W(r) = -|S| r^(dim-1) G'(r) = kr [K1(kr) + K0(kR) I1(kr)/I0(kR)] (2D),
 * [kr cosh(k(R - r)) + sinh(k(R - r))] / sinh kR (3D), which is C at r = R
 * and 1 as r -> 0 (Green's identity on the star-shaped region, whose
 * boundary elements seen from x under the solid angle dw have
 * n . (z - x) / r dz = r^(dim-1) dw).  A step's source and Neumann terms use
 * G in place of the Laplace ball's Green's function (the source sample at
 * rho = r u2: -|S| r rho^(dim-1) G(rho)), weighted by the product of the
 * factors of the steps before it; the gradient of a start inside the domain
 * is (dim/R0) Qg [(U - w_f0)/C - cv] nu + w_g0, as wos_estimate_sigma. */
bvc_status bvc_mixed_walk_sigma(bvc_mixed m, const bvc_function* gfn, const bvc_neumann* h, const bvc_function* ffn,
                                double sigma, const float* starts, const int32_t* start_elem, const float* nrm,
                                int64_t n, int32_t walks, float eps, int32_t max_steps, uint64_t seed, uint64_t id_base,
                                uint32_t tag, float* rec, int32_t* steps, int32_t* prim, unsigned long long* counter,
                                bvc_stream stream);

/* The mixed cache: K1 on the whole boundary (Neumann samples at offset 0,
 * Dirichlet samples on the Dirichlet offset boundary at offset_l), walks on
 * stars (tag 0, ids as bvc_cache_build), K3, source samples (opts->src_grid,
 * inside the whole boundary itself), pack.  dudn_hat of a Neumann sample is h(z).
 * opts->sigma > 0: the screened walks of bvc_mixed_walk_sigma, and the cache
 * records sigma so that bvc_evaluate uses the screened Green's functions of
 * App. A.  clamp_c must be 0 (BVC_ERR_UNSUPPORTED otherwise).  Workspace as
 * bvc_cache_build on the whole geometry. */
bvc_status bvc_mixed_cache_build_workspace_size(bvc_mixed m, const bvc_cache_opts* opts, size_t* min_bytes,
                                                size_t* full_bytes);
bvc_status bvc_mixed_cache_build(bvc_mixed m, const bvc_function* gfn, const bvc_neumann* h, const bvc_function* ffn,
                                 const bvc_cache_opts* opts, bvc_cache* cache, void* workspace,
                                 size_t workspace_bytes, bvc_stream stream);

/* Pointwise walk on stars at the points of `state` (tag 3), as wos_estimate:
 * u_bnd += sum_j U, grad_bnd += sum_j grad (if set), counts[0] += walks.
 * Workspace: wos_estimate_workspace_size. */
bvc_status wost_estimate(bvc_mixed m, const bvc_function* gfn, const bvc_neumann* h, const bvc_function* ffn,
                         bvc_eval_state* state, int32_t walks, float eps, int32_t max_steps, uint64_t seed,
                         uint64_t id_base, void* workspace, size_t workspace_bytes, bvc_stream stream);
/* wost_estimate for the screened equation (Delta - sigma) u = f (sigma >= 0;
 * the walks of bvc_mixed_walk_sigma).  sigma = 0 is wost_estimate. */
bvc_status wost_estimate_sigma(bvc_mixed m, const bvc_function* gfn, const bvc_neumann* h, const bvc_function* ffn,
                               double sigma, bvc_eval_state* state, int32_t walks, float eps, int32_t max_steps,
                               uint64_t seed, uint64_t id_base, void* workspace, size_t workspace_bytes,
                               bvc_stream stream);

/* ------------------------------------------------------------- profiling */
/* Between bvc_profile_begin and bvc_profile_end every kernel the library
 * launches is bracketed by CUDA events on its own stream.  bvc_profile_end
 * waits for them and returns per-kernel totals (launch count, summed
 * duration), at most max_out entries.  Not thread-safe: profile one host
 * thread's calls at a time. */
typedef struct {
  char name[32];
  int64_t launches;
  double total_ms;
} bvc_kernel_time;
bvc_status bvc_profile_begin(void);
bvc_status bvc_profile_end(bvc_kernel_time* out, int32_t max_out, int32_t* n_out);

/* ------------------------------------------------------------------ misc */
const char* bvc_status_string(bvc_status s);
/* The last status other than BVC_OK that any entry point returned on the
 * calling thread (thread-local; every call returns its status directly as
 * well), or BVC_OK if there was none since the previous bvc_last_error call;
 * the call clears it.  Device-side conditions are read per handle
 * (bvc_geometry_stats, bvc_batch_stats, bvc_gather_status) and also pass
 * through here when those calls return them. */
bvc_status bvc_last_error(void);
/* Library version as major*10000 + minor*100 + patch. */
int32_t bvc_version(void);

/* ----------------------------------------------------------- debug build */
/* A debug build of the library (compiled with BVC_DEBUG=1) checks, in every
 * BVH traversal on the device (closest point, ray, silhouette, Neumann
 * descent), each node index against the tree size, each leaf's primitive
 * range against the primitive count and each traversal stack push against
 * the stack depth, before the access.  A failed check skips the access,
 * sets bit 1 of the geometry's status flags and lets the kernel finish;
 * bvc_geometry_stats (bvc_batch_stats for a forest) then returns
 * BVC_ERR_BOUNDS.  Release builds compile the checks out.
 * bvc_debug_build returns 1 in a debug build, 0 otherwise. */
int32_t bvc_debug_build(void);
/* Test hook of the debug build: overwrites child `side` (0 left, 1 right)
 * of internal node `node` of g's BVH with the raw link `link` (>= 0 an
 * internal node index, < 0 the complement of a leaf's (first << 4) | count)
 * on `stream`; the host copy of the tree is not changed.  Used to check that
 * a corrupted link is caught: the library never writes a link that the
 * checks above would reject.  Release builds: BVC_ERR_UNSUPPORTED, nothing
 * written.  node outside [0, n_nodes) or side not 0/1: BVC_ERR_INVALID_ARG. */
bvc_status bvc_debug_set_link(bvc_geometry g, int64_t node, int32_t side, int32_t link, bvc_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* BVC_H_ */
