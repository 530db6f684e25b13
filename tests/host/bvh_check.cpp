// Structural check of the host BVH builder (paper_2302_11825_gb300/csrc/
// bvh_build.cpp), built with AddressSanitizer and UBSan by the CPU tests.
// Reads a mesh (int32 dim, int64 n_verts, int64 n_prims, float32 V[n_verts*dim],
// int32 F[n_prims*dim]) and checks the flattened tree the walk kernels
// traverse: every primitive in exactly one leaf, the caller ids a
// permutation, children after their parent, depth within the traversal
// stack, leaf counts within the 4-bit encoding, every stored child box
// containing what lies below it, and every child slab (unit normal n,
// [dmin, dmax]) holding n . v of every vertex below it (or unbounded).
// Prints one line; exit status 0 = all good.
#include <vector_types.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

namespace bvc {
int64_t build_bvh(int dim, const float* V, const int32_t* F, int64_t np, std::vector<float4>& nodes_out,
                  std::vector<float4>& prims_out, std::vector<int32_t>& ids_out, std::vector<float4>* slabs_out);
}

namespace {

struct Ctx {
  int dim = 0, per = 0;
  std::vector<float> V;
  std::vector<int32_t> F;
  std::vector<float4> nodes;
  std::vector<float4> slabs;
  std::vector<int32_t> ids;
  std::vector<int> seen;
  int max_depth = 0, bad_order = 0, bad_box = 0, bad_count = 0;
  int64_t bad_slab = 0, unbounded = 0, slabbed = 0;
};

// Slab of child k of a node: unit normal (zero = unbounded) and interval.
void child_slab(const Ctx& c, int64_t node, int k, float* n, float* dmin, float* dmax) {
  const float4* q = &c.slabs[node * (c.dim == 2 ? 2 : 3)];
  if (c.dim == 2) {
    n[0] = q[k].x, n[1] = q[k].y, n[2] = 0.0f, *dmin = q[k].z, *dmax = q[k].w;
  } else if (k == 0) {
    n[0] = q[0].x, n[1] = q[0].y, n[2] = q[0].z, *dmin = q[0].w, *dmax = q[1].x;
  } else {
    n[0] = q[1].y, n[1] = q[1].z, n[2] = q[1].w, *dmin = q[2].x, *dmax = q[2].y;
  }
}

// Elements below child encoding ch (appended to out).
void collect(const Ctx& c, int32_t ch, std::vector<int32_t>& out) {
  if (ch < 0) {
    const int32_t enc = ~ch, first = enc >> 4, count = enc & 15;
    for (int32_t q = first; q < first + count && q < (int32_t)c.ids.size(); ++q) out.push_back(c.ids[q]);
    return;
  }
  for (int k = 0; k < 2; ++k) {
    int32_t gc;
    std::memcpy(&gc, (const char*)&c.nodes[(int64_t)ch * c.per + c.per - 1] + 4 * k, 4);
    collect(c, gc, out);
  }
}

// Every child slab of every node holds the vertices of the elements below it.
void check_slabs(Ctx& c, int64_t node) {
  for (int k = 0; k < 2; ++k) {
    int32_t gc;
    std::memcpy(&gc, (const char*)&c.nodes[node * c.per + c.per - 1] + 4 * k, 4);
    float n[3], dmin, dmax;
    child_slab(c, node, k, n, &dmin, &dmax);
    const double nl = std::sqrt((double)n[0] * n[0] + (double)n[1] * n[1] + (double)n[2] * n[2]);
    if (nl == 0.0) {
      ++c.unbounded;
      if (!(dmin <= -1e38f && dmax >= 1e38f)) ++c.bad_slab;
    } else {
      ++c.slabbed;
      if (std::fabs(nl - 1.0) > 1e-6) ++c.bad_slab;
      std::vector<int32_t> el;
      collect(c, gc, el);
      for (int32_t e : el)
        for (int v = 0; v < c.dim; ++v) {
          const float* p = &c.V[(int64_t)c.F[(int64_t)e * c.dim + v] * c.dim];
          double d = 0.0;
          for (int a = 0; a < c.dim; ++a) d += (double)n[a] * p[a];
          if (!(d >= dmin && d <= dmax)) ++c.bad_slab;
        }
    }
    if (gc >= 0) check_slabs(c, gc);
  }
}

void child_box(const Ctx& c, int64_t node, int k, float* lo, float* hi) {
  const float4* n = &c.nodes[node * c.per];
  if (c.dim == 2) {
    const float4 b = n[k];
    lo[0] = b.x, lo[1] = b.y, hi[0] = b.z, hi[1] = b.w;
    lo[2] = hi[2] = 0.0f;
  } else if (k == 0) {
    lo[0] = n[0].x, lo[1] = n[0].y, lo[2] = n[0].z, hi[0] = n[0].w, hi[1] = n[1].x, hi[2] = n[1].y;
  } else {
    lo[0] = n[1].z, lo[1] = n[1].w, lo[2] = n[2].x, hi[0] = n[2].y, hi[1] = n[2].z, hi[2] = n[2].w;
  }
}

bool inside(const float* lo, const float* hi, const float* p, int dim) {
  for (int a = 0; a < dim; ++a)
    if (!(p[a] >= lo[a] && p[a] <= hi[a])) return false;
  return true;
}

// Visits the subtree `ch` whose box (stored in its parent) is [lo, hi].
void visit(Ctx& c, int64_t parent, int32_t ch, const float* lo, const float* hi, int depth) {
  if (depth > c.max_depth) c.max_depth = depth;
  if (ch < 0) {
    const int32_t enc = ~ch, first = enc >> 4, count = enc & 15;
    if (count < 0 || count > 15 || first < 0 || first + count > (int32_t)c.seen.size()) {
      ++c.bad_count;
      return;
    }
    for (int32_t q = first; q < first + count; ++q) {
      ++c.seen[q];
      const int32_t e = c.ids[q];
      for (int v = 0; v < c.dim; ++v)
        if (!inside(lo, hi, &c.V[(int64_t)c.F[(int64_t)e * c.dim + v] * c.dim], c.dim)) ++c.bad_box;
    }
    return;
  }
  if ((int64_t)ch <= parent || (int64_t)ch * c.per >= (int64_t)c.nodes.size()) {
    ++c.bad_order;
    return;
  }
  for (int k = 0; k < 2; ++k) {
    float clo[3], chi[3];
    child_box(c, ch, k, clo, chi);
    int32_t gc;
    std::memcpy(&gc, (const char*)&c.nodes[(int64_t)ch * c.per + c.per - 1] + 4 * k, 4);
    // an empty child (a root with a single leaf) has an inverted box and no primitives
    const bool empty = gc < 0 && ((~gc) & 15) == 0;
    if (!empty)
      for (int a = 0; a < c.dim; ++a)
        if (!(clo[a] >= lo[a] && chi[a] <= hi[a])) ++c.bad_box;
    visit(c, ch, gc, clo, chi, depth + 1);
  }
}

}  // namespace

int main(int argc, char** argv) {
  if (argc != 2) return 2;
  FILE* f = std::fopen(argv[1], "rb");
  if (!f) return 2;
  Ctx c;
  int32_t dim = 0;
  int64_t nv = 0, np = 0;
  bool ok = std::fread(&dim, 4, 1, f) == 1 && std::fread(&nv, 8, 1, f) == 1 && std::fread(&np, 8, 1, f) == 1 &&
            (dim == 2 || dim == 3) && nv > 0 && np > 0;
  if (ok) {
    c.V.resize(nv * dim);
    c.F.resize(np * dim);
    ok = std::fread(c.V.data(), 4, nv * dim, f) == (size_t)(nv * dim) &&
         std::fread(c.F.data(), 4, np * dim, f) == (size_t)(np * dim);
  }
  std::fclose(f);
  if (!ok) return 2;
  c.dim = dim;
  c.per = dim == 2 ? 3 : 4;
  std::vector<float4> prims;
  const int64_t nn = bvc::build_bvh(dim, c.V.data(), c.F.data(), np, c.nodes, prims, c.ids, &c.slabs);
  c.seen.assign(np, 0);
  const float big = INFINITY;
  const float lo[3] = {-big, -big, -big}, hi[3] = {big, big, big};
  // the root (node 0) is internal: visit its two children
  for (int k = 0; k < 2; ++k) {
    float clo[3], chi[3];
    child_box(c, 0, k, clo, chi);
    int32_t gc;
    std::memcpy(&gc, (const char*)&c.nodes[c.per - 1] + 4 * k, 4);
    (void)lo;
    (void)hi;
    visit(c, 0, gc, clo, chi, 1);
  }
  int64_t not_once = 0;
  for (int s : c.seen) not_once += s != 1;
  std::vector<int> idc(np, 0);
  int64_t bad_ids = 0;
  for (int32_t e : c.ids) {
    if (e < 0 || e >= np) ++bad_ids;
    else ++idc[e];
  }
  for (int s : idc) bad_ids += s != 1;
  const bool slabs_sized = (int64_t)c.slabs.size() == nn * (dim == 2 ? 2 : 3);
  if (slabs_sized) check_slabs(c, 0);
  std::printf("dim=%d prims=%lld nodes=%lld max_depth=%d not_once=%lld bad_ids=%lld bad_order=%d bad_box=%d "
              "bad_count=%d slabs=%lld unbounded=%lld bad_slab=%lld\n",
              dim, (long long)np, (long long)nn, c.max_depth, (long long)not_once, (long long)bad_ids, c.bad_order,
              c.bad_box, c.bad_count, (long long)c.slabbed, (long long)c.unbounded, (long long)c.bad_slab);
  const bool good = nn * c.per == (int64_t)c.nodes.size() && c.max_depth <= 24 && not_once == 0 && bad_ids == 0 &&
                    c.bad_order == 0 && c.bad_box == 0 && c.bad_count == 0 && slabs_sized && c.bad_slab == 0;
  return good ? 0 : 1;
}
