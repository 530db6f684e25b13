// bvc_common.cu -- host helpers: problem-function conversion, device
// properties, status strings.
#include <nvtx3/nvToolsExt.h>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "bvc_internal.h"

namespace bvc {

bool make_dev_function(const bvc_function* f, int dim, DevFunction* out) {
  *out = DevFunction{};
  if (f == nullptr || f->n_terms == 0) return true;
  if (f->n_terms < 0 || f->n_terms > BVC_MAX_TERMS) return false;
  int used = 0;
  out->n_terms = f->n_terms;
  for (int t = 0; t < f->n_terms; ++t) {
    const bvc_term& tm = f->terms[t];
    const int nc = tm.n_coeffs;
    if (nc < 0 || (nc > 0 && tm.coeffs == nullptr)) return false;
    for (int i = 0; i < nc; ++i)
      if (!std::isfinite(tm.coeffs[i])) return false;
    out->kind[t] = tm.kind;
    out->off[t] = used;
    float* c = out->c + used;
    int dn = nc;
    switch (tm.kind) {
      case BVC_FN_POLY:
        if (nc > (dim == 2 ? 15 : 35)) return false;
        if (used + nc > BVC_MAX_COEFFS) return false;
        for (int i = 0; i < nc; ++i) c[i] = (float)tm.coeffs[i];
        break;
      case BVC_FN_GAUSS:
      case BVC_FN_GAUSS_LAPLACIAN: {
        if (nc < 1 || (nc - 1) % (1 + dim) != 0) return false;
        const double s = tm.coeffs[0];
        if (!(s > 0.0)) return false;
        const int head = tm.kind == BVC_FN_GAUSS ? 1 : 3;
        dn = head + (nc - 1);
        if (used + dn > BVC_MAX_COEFFS + 8) return false;
        c[0] = (float)(-1.0 / (2.0 * s * s));
        if (head == 3) {
          c[1] = (float)(1.0 / (s * s * s * s));
          c[2] = (float)(-(double)dim / (s * s));
        }
        for (int i = 1; i < nc; ++i) c[head + i - 1] = (float)tm.coeffs[i];
        break;
      }
      case BVC_FN_EXP_TRIG:
        if (dim != 3 || nc != 4) return false;
        if (used + nc > BVC_MAX_COEFFS) return false;
        for (int i = 0; i < 4; ++i) c[i] = (float)tm.coeffs[i];
        break;
      case BVC_FN_EXP_COS:
        if (nc != 3) return false;
        if (used + nc > BVC_MAX_COEFFS) return false;
        for (int i = 0; i < 3; ++i) c[i] = (float)tm.coeffs[i];
        break;
      default:
        return false;
    }
    out->nc[t] = dn;
    used += dn;
  }
  return true;
}

int num_sms() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (dev < 0 || dev >= 64) return 1;
  if (cached[dev] == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
    cached[dev] = n;
  }
  return cached[dev];
}

int max_blocks_per_sm(const void* kernel, int block, size_t smem) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, block, smem) != cudaSuccess || n <= 0) n = 1;
  return n;
}

namespace {
struct ProfRec {
  const char* name;
  cudaEvent_t a, b;
};
struct Profiler {
  std::mutex mu;
  bool on = false;
  std::vector<ProfRec> recs;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
  }
};
Profiler& prof() {
  static Profiler p;
  return p;
}
}  // namespace

ProfScope::ProfScope(const char* name, cudaStream_t s) : slot_(-1), s_(s) {
  // an NVTX range around every launch, named for its step (K1 sample_boundary,
  // K2/K6 walk, K3 reduce_walks, K4 source_*, K5 gather_*, ...), for
  // timeline tools; without a tool attached the call returns at once
  nvtxRangePushA(name);
  Profiler& P = prof();
  std::lock_guard<std::mutex> g(P.mu);
  if (!P.on) return;
  ProfRec r{name, P.get(), P.get()};
  if (r.a == nullptr || r.b == nullptr) return;
  if (cudaEventRecord(r.a, s) != cudaSuccess) return;
  slot_ = (int)P.recs.size();
  P.recs.push_back(r);
}

ProfScope::~ProfScope() {
  nvtxRangePop();
  if (slot_ < 0) return;
  Profiler& P = prof();
  std::lock_guard<std::mutex> g(P.mu);
  if (slot_ < (int)P.recs.size()) cudaEventRecord(P.recs[slot_].b, s_);
}

}  // namespace bvc

static bvc_status bvc_profile_begin_impl(void) {
  bvc::Profiler& P = bvc::prof();
  std::lock_guard<std::mutex> g(P.mu);
  for (auto& r : P.recs) {
    P.pool.push_back(r.a);
    P.pool.push_back(r.b);
  }
  P.recs.clear();
  P.on = true;
  return BVC_OK;
}
extern "C" bvc_status bvc_profile_begin(void) {
  return bvc::note_status(bvc_profile_begin_impl());
}

static bvc_status bvc_profile_end_impl(bvc_kernel_time* out, int32_t max_out, int32_t* n_out) {
  bvc::Profiler& P = bvc::prof();
  std::lock_guard<std::mutex> g(P.mu);
  P.on = false;
  int32_t n = 0;
  bvc_status st = BVC_OK;
  for (auto& r : P.recs) {
    if (cudaEventSynchronize(r.b) != cudaSuccess) {
      st = BVC_ERR_CUDA;
      continue;
    }
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) {
      st = BVC_ERR_CUDA;
      continue;
    }
    int32_t k = 0;
    while (k < n && std::strncmp(out[k].name, r.name, sizeof(out[k].name)) != 0) ++k;
    if (k == n) {
      if (out == nullptr || n >= max_out) continue;
      std::memset(&out[k], 0, sizeof(out[k]));
      std::strncpy(out[k].name, r.name, sizeof(out[k].name) - 1);
      ++n;
    }
    out[k].launches += 1;
    out[k].total_ms += ms;
  }
  for (auto& r : P.recs) {
    P.pool.push_back(r.a);
    P.pool.push_back(r.b);
  }
  P.recs.clear();
  if (n_out) *n_out = n;
  (void)cudaGetLastError();
  return st;
}
extern "C" bvc_status bvc_profile_end(bvc_kernel_time* out, int32_t max_out, int32_t* n_out) {
  return bvc::note_status(bvc_profile_end_impl(out, max_out, n_out));
}

extern "C" const char* bvc_status_string(bvc_status s) {
  switch (s) {
    case BVC_OK: return "ok";
    case BVC_ERR_INVALID_ARG: return "invalid argument";
    case BVC_ERR_DEGENERATE_MESH: return "degenerate mesh";
    case BVC_ERR_OOM: return "out of device memory";
    case BVC_ERR_CUDA: return "CUDA runtime error";
    case BVC_ERR_TIMEOUT: return "in-kernel wait timed out";
    case BVC_ERR_UNSUPPORTED: return "unsupported";
    case BVC_ERR_WORKSPACE: return "workspace too small";
    case BVC_WARN_WALK_CAP: return "walks stopped at max_steps";
    case BVC_ERR_BOUNDS: return "device bounds check failed (debug build)";
  }
  return "unknown status";
}

extern "C" int32_t bvc_version(void) { return 100; }

namespace bvc {
thread_local bvc_status g_last_status = BVC_OK;
}

extern "C" bvc_status bvc_last_error(void) {
  const bvc_status s = bvc::g_last_status;
  bvc::g_last_status = BVC_OK;
  return s;
}
