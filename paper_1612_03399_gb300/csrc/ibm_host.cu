// Host side of the C ABI: input validation, the mesh auxiliary arrays of
// Sec. 5 (edges, faces of each edge, the four vertices of each hinge, vertex
// incidence), per-patch tables of the force kernel, the rest state in float64,
// device upload and the entry points declared in include/ibm.h.
#include <cuda_runtime.h>
#include <cstdlib>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <initializer_list>
#include <unordered_map>
#include <utility>
#include <vector>

#include "ibm_internal.cuh"

using namespace ibm;

namespace {

std::mutex g_mu;
std::string g_err;

struct Failure {
  ibm_status s;
  std::string msg;
};

[[noreturn]] void fail(ibm_status s, const std::string& m) { throw Failure{s, m}; }

void check_cuda(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    fail(e == cudaErrorMemoryAllocation ? IBM_ERR_OOM : IBM_ERR_CUDA,
         std::string(what) + ": " + cudaGetErrorString(e));
  }
}

struct HostTopo {
  int nv = 0, nf = 0, ne = 0;
  bool has_boundary = false;
  std::vector<int32_t> tri;
  std::vector<int4> edge;  // a, b, c, d
  std::vector<int2> eface; // face holding a->b, face holding b->a (-1 if none)
  std::vector<int32_t> v2f_ptr, v2f_idx;
  std::vector<PatchHdr> patch;
  std::vector<int32_t> loc_vert;
  std::vector<PEdge> pedge;
  std::vector<PFace> pface;
  std::vector<int32_t> csr_ptr;
  std::vector<uint16_t> csr_slot;
  std::vector<uint32_t> fblob;          // packed element records of the force kernel
  std::vector<FPatch> fpatch;           //   (one 16-byte aligned blob per patch)
  std::vector<int32_t> fatt;            // per face: 2 * attached edge + side (1: right face)
  std::vector<int32_t> fface;           // per patch, its faces in the blob's order
  int max_loc = 0, max_slot = 0, max_own = 0;
  std::vector<int32_t> mface, mbound;   // faces in marker-patch order, patch boundaries
};

inline uint64_t key2(int32_t p, int32_t q) {
  return ((uint64_t)(uint32_t)p << 32) | (uint32_t)q;
}

// Edges, hinges and incidence of one oriented triangle mesh, plus the patch
// tables.  Throws IBM_ERR_MESH on index errors, repeated vertices in a face,
// a directed edge used twice (an edge shared by more than two faces or two
// faces of opposite orientation).
void build_topology(HostTopo& T, const int32_t* tri, int nv, int nf, int P) {
  T.nv = nv;
  T.nf = nf;
  T.tri.assign(tri, tri + 3 * (size_t)nf);
  std::unordered_map<uint64_t, int32_t> half, hface;
  half.reserve((size_t)nf * 6);
  hface.reserve((size_t)nf * 6);
  for (int f = 0; f < nf; ++f) {
    const int a = tri[3 * f], b = tri[3 * f + 1], c = tri[3 * f + 2];
    if (a < 0 || b < 0 || c < 0 || a >= nv || b >= nv || c >= nv)
      fail(IBM_ERR_MESH, "face " + std::to_string(f) + " has a vertex index out of range");
    if (a == b || b == c || c == a)
      fail(IBM_ERR_MESH, "face " + std::to_string(f) + " repeats a vertex");
    const int hp[3][3] = {{a, b, c}, {b, c, a}, {c, a, b}};
    for (auto& h : hp) {
      hface.emplace(key2(h[0], h[1]), f);
      if (!half.emplace(key2(h[0], h[1]), h[2]).second)
        fail(IBM_ERR_MESH, "edge (" + std::to_string(h[0]) + "," + std::to_string(h[1]) +
                               ") is used twice in the same direction: non-manifold or "
                               "inconsistently oriented mesh");
    }
  }
  std::unordered_map<uint64_t, int32_t> und;
  und.reserve((size_t)nf * 3);
  for (int f = 0; f < nf; ++f) {
    const int a = tri[3 * f], b = tri[3 * f + 1], c = tri[3 * f + 2];
    const int hp[3][3] = {{a, b, c}, {b, c, a}, {c, a, b}};
    for (auto& h : hp) {
      const uint64_t k = key2(std::min(h[0], h[1]), std::max(h[0], h[1]));
      if (und.count(k)) continue;
      auto it = half.find(key2(h[1], h[0]));
      const int s = it == half.end() ? -1 : it->second;
      if (s < 0) T.has_boundary = true;
      und.emplace(k, (int32_t)T.edge.size());
      T.edge.push_back(make_int4(h[0], h[1], h[2], s));
      const auto jt = hface.find(key2(h[1], h[0]));
      T.eface.push_back(make_int2(f, jt == hface.end() ? -1 : jt->second));
    }
  }
  T.ne = (int)T.edge.size();
  // vertex -> face
  T.v2f_ptr.assign(nv + 1, 0);
  for (int f = 0; f < nf; ++f)
    for (int k = 0; k < 3; ++k) T.v2f_ptr[tri[3 * f + k] + 1]++;
  for (int v = 0; v < nv; ++v) T.v2f_ptr[v + 1] += T.v2f_ptr[v];
  T.v2f_idx.assign(T.v2f_ptr[nv], 0);
  std::vector<int32_t> fill(T.v2f_ptr.begin(), T.v2f_ptr.end() - 1);
  std::vector<int32_t> v2fc(T.v2f_ptr[nv]);  // face*3 + corner
  for (int f = 0; f < nf; ++f)
    for (int k = 0; k < 3; ++k) {
      const int v = tri[3 * f + k];
      v2fc[fill[v]] = 3 * f + k;
      T.v2f_idx[fill[v]++] = f;
    }
  // vertex -> (edge, role) with role 0..3 = a, b, c, d
  std::vector<int32_t> v2e_ptr(nv + 1, 0);
  for (const int4& e : T.edge) {
    v2e_ptr[e.x + 1]++;
    v2e_ptr[e.y + 1]++;
    v2e_ptr[e.z + 1]++;
    if (e.w >= 0) v2e_ptr[e.w + 1]++;
  }
  for (int v = 0; v < nv; ++v) v2e_ptr[v + 1] += v2e_ptr[v];
  std::vector<int32_t> v2e(v2e_ptr[nv]);
  fill.assign(v2e_ptr.begin(), v2e_ptr.end() - 1);
  for (int e = 0; e < T.ne; ++e) {
    const int4 E = T.edge[e];
    v2e[fill[E.x]++] = 4 * e + 0;
    v2e[fill[E.y]++] = 4 * e + 1;
    v2e[fill[E.z]++] = 4 * e + 2;
    if (E.w >= 0) v2e[fill[E.w]++] = 4 * e + 3;
  }
  // face -> edge attachment of the force kernel: a matching in which every
  // face holds an edge of its own (it exists: a set of k faces touches at
  // least 3k/2 edges, each edge having at most two faces), preferring the
  // edges of which the face is the left face; the rest by augmenting paths.
  {
    std::vector<int32_t> fe(3 * (size_t)nf);
    for (int f = 0; f < nf; ++f)
      for (int k = 0; k < 3; ++k) {
        const int p0 = tri[3 * f + k], p1 = tri[3 * f + (k + 1) % 3];
        fe[3 * f + k] = und.at(key2(std::min(p0, p1), std::max(p0, p1)));
      }
    std::vector<int32_t> owner(T.ne, -1), fedge(nf, -1);
    for (int e = 0; e < T.ne; ++e) {
      const int f = T.eface[e].x;
      if (fedge[f] < 0) { fedge[f] = e; owner[e] = f; }
    }
    for (int e = 0; e < T.ne; ++e) {
      const int f = T.eface[e].y;
      if (f >= 0 && fedge[f] < 0 && owner[e] < 0) { fedge[f] = e; owner[e] = f; }
    }
    std::vector<int32_t> seen(nf, -1), from(nf, -1), via(nf, -1), queue;
    for (int f0 = 0; f0 < nf; ++f0) {
      if (fedge[f0] >= 0) continue;
      // breadth-first search for a free edge along alternating paths
      queue.assign(1, f0);
      seen[f0] = f0;
      int end_f = -1, end_e = -1;
      for (size_t qi = 0; qi < queue.size() && end_f < 0; ++qi) {
        const int f = queue[qi];
        for (int k = 0; k < 3 && end_f < 0; ++k) {
          const int e = fe[3 * f + k];
          if (owner[e] < 0) {
            end_f = f;
            end_e = e;
          } else if (seen[owner[e]] != f0) {
            seen[owner[e]] = f0;
            from[owner[e]] = f;
            via[owner[e]] = e;
            queue.push_back(owner[e]);
          }
        }
      }
      if (end_f < 0) fail(IBM_ERR_MESH, "no face-edge matching (non-manifold mesh)");
      // flip the path: each face on it takes the edge that led to its successor
      int f = end_f, e = end_e;
      while (true) {
        const int prev_e = fedge[f];
        fedge[f] = e;
        owner[e] = f;
        if (f == f0) break;
        e = via[f];   // == prev_e: the edge f held, now passed to its predecessor
        (void)prev_e;
        f = from[f];
      }
    }
    T.fatt.assign(nf, -1);
    for (int f = 0; f < nf; ++f) {
      const int e = fedge[f];
      if (e < 0 || owner[e] != f || (fe[3 * f] != e && fe[3 * f + 1] != e && fe[3 * f + 2] != e))
        fail(IBM_ERR_MESH, "face-edge matching failed");
      T.fatt[f] = 2 * e + (T.eface[e].x == f ? 0 : 1);
    }
  }
  // patches
  const int npatch = (nv + P - 1) / P;
  std::vector<int32_t> e_stamp(T.ne, -1), e_loc(T.ne), f_stamp(nf, -1), f_loc(nf),
      v_stamp(nv, -1), v_loc(nv);
  std::vector<int32_t> es, fs;
  for (int p = 0; p < npatch; ++p) {
    PatchHdr H{};
    const int o0 = p * P, o1 = std::min(nv, o0 + P);
    H.own0 = o0;
    H.n_own = o1 - o0;
    H.loc_off = (int32_t)T.loc_vert.size();
    for (int v = o0; v < o1; ++v) {
      v_stamp[v] = p;
      v_loc[v] = v - o0;
      T.loc_vert.push_back(v);
    }
    auto local = [&](int v) -> uint16_t {
      if (v < 0) return kNone;
      if (v_stamp[v] != p) {
        v_stamp[v] = p;
        v_loc[v] = (int32_t)T.loc_vert.size() - H.loc_off;
        T.loc_vert.push_back(v);
      }
      return (uint16_t)v_loc[v];
    };
    es.clear();
    fs.clear();
    for (int v = o0; v < o1; ++v) {
      for (int k = v2e_ptr[v]; k < v2e_ptr[v + 1]; ++k) {
        const int e = v2e[k] >> 2;
        if (e_stamp[e] != p) {
          e_stamp[e] = p;
          es.push_back(e);
        }
      }
      for (int k = T.v2f_ptr[v]; k < T.v2f_ptr[v + 1]; ++k) {
        const int f = T.v2f_idx[k];
        if (f_stamp[f] != p) {
          f_stamp[f] = p;
          fs.push_back(f);
        }
      }
    }
    std::sort(es.begin(), es.end());
    std::sort(fs.begin(), fs.end());
    H.edge_off = (int32_t)T.pedge.size();
    H.n_edge = (int32_t)es.size();
    for (size_t i = 0; i < es.size(); ++i) {
      const int e = es[i];
      e_loc[e] = (int32_t)i;
      const int4 E = T.edge[e];
      PEdge r;
      r.l[0] = local(E.x);
      r.l[1] = local(E.y);
      r.l[2] = local(E.z);
      r.l[3] = local(E.w);
      r.eid = e | ((E.x >= o0 && E.x < o1) ? (int32_t)0x80000000 : 0);
      T.pedge.push_back(r);
    }
    H.face_off = (int32_t)T.pface.size();
    H.n_face = (int32_t)fs.size();
    for (size_t i = 0; i < fs.size(); ++i) {
      const int f = fs[i];
      f_loc[f] = (int32_t)i;
      PFace r;
      r.l[0] = local(tri[3 * f]);
      r.l[1] = local(tri[3 * f + 1]);
      r.l[2] = local(tri[3 * f + 2]);
      r.owned = (tri[3 * f] >= o0 && tri[3 * f] < o1) ? 1 : 0;
      r.fid = f;
      T.pface.push_back(r);
    }
    H.n_loc = (int32_t)T.loc_vert.size() - H.loc_off;
    H.n_slot = 4 * H.n_edge + 3 * H.n_face;
    if (H.n_loc >= (int)kNone || H.n_slot > 65535)
      fail(IBM_ERR_UNSUPPORTED, "patch too large for 16-bit local indices; lower patch_size");
    H.csr_off = (int32_t)T.csr_ptr.size();
    H.slot_off = (int32_t)T.csr_slot.size();
    for (int v = o0; v < o1; ++v) {
      T.csr_ptr.push_back((int32_t)T.csr_slot.size() - H.slot_off);
      // contribution slots are laid out [role][element] (edges, then faces)
      for (int k = v2e_ptr[v]; k < v2e_ptr[v + 1]; ++k) {
        const int e = v2e[k] >> 2, role = v2e[k] & 3;
        T.csr_slot.push_back((uint16_t)(role * H.n_edge + e_loc[e]));
      }
      for (int k = T.v2f_ptr[v]; k < T.v2f_ptr[v + 1]; ++k) {
        const int f = v2fc[k] / 3, corner = v2fc[k] % 3;
        T.csr_slot.push_back((uint16_t)(4 * H.n_edge + corner * H.n_face + f_loc[f]));
      }
    }
    T.csr_ptr.push_back((int32_t)T.csr_slot.size() - H.slot_off);
    // The force kernel's blob of this patch.  Every face is attached to an
    // edge of its own (as its left face (a, b, c) or its right face (b, a, d))
    // and adds its corner forces to that edge's role slots, so an own vertex
    // has one slot per edge role it plays, contiguous and in the order of its
    // edge list above.  Per edge 4 words (a | b << 16, c | d << 16, slot of a |
    // slot of b << 16, slot of c | slot of d << 16; kNone for halo vertices);
    // per face 2 words (edge | side << 30 | owned << 31, face id); then the
    // first slot of every own vertex (n_own + 1 16-bit entries).
    {
      std::vector<uint16_t> dE(4 * es.size(), kNone);
      std::vector<int32_t> ptr(H.n_own + 1);
      int32_t n = 0;
      for (int v = o0; v < o1; ++v) {
        ptr[v - o0] = n;
        for (int k = v2e_ptr[v]; k < v2e_ptr[v + 1]; ++k)
          dE[4 * e_loc[v2e[k] >> 2] + (v2e[k] & 3)] = (uint16_t)n++;
      }
      ptr[H.n_own] = n;
      if (n >= (int)kNone)
        fail(IBM_ERR_UNSUPPORTED, "patch too large for 16-bit local indices; lower patch_size");
      FPatch Q{};
      Q.blob_off = (int32_t)T.fblob.size();
      Q.n_slot = n;
      for (size_t i = 0; i < es.size(); ++i) {
        const PEdge& r = T.pedge[H.edge_off + i];
        T.fblob.push_back(r.l[0] | (uint32_t)r.l[1] << 16);
        T.fblob.push_back(r.l[2] | (uint32_t)r.l[3] << 16);
        T.fblob.push_back(dE[4 * i] | (uint32_t)dE[4 * i + 1] << 16);
        T.fblob.push_back(dE[4 * i + 2] | (uint32_t)dE[4 * i + 3] << 16);
      }
      // faces in the patch's order; their rest data follows the same order
      const std::vector<int32_t>& fo = fs;
      for (const int f : fo) {
        const int e = T.fatt[f] >> 1;
        if (e_stamp[e] != p) fail(IBM_ERR_MESH, "face attached to an edge outside its patch");
        const bool owned = tri[3 * f] >= o0 && tri[3 * f] < o1;
        T.fblob.push_back((uint32_t)e_loc[e] | (uint32_t)(T.fatt[f] & 1) << 30 |
                          (owned ? 0x80000000u : 0u));
        T.fblob.push_back((uint32_t)f);
      }
      for (size_t i = 0; i < ptr.size(); i += 2)
        T.fblob.push_back((uint32_t)ptr[i] | (i + 1 < ptr.size() ? (uint32_t)ptr[i + 1] << 16 : 0u));
      while (T.fblob.size() % 4) T.fblob.push_back(0u);
      Q.blob_words = (int32_t)T.fblob.size() - Q.blob_off;
      // adjoint-only tail: the faces of each own vertex with its corner
      std::vector<int32_t> vptr(H.n_own + 1);
      std::vector<uint32_t> vent;
      for (int v = o0; v < o1; ++v) {
        vptr[v - o0] = (int32_t)vent.size();
        for (int k = T.v2f_ptr[v]; k < T.v2f_ptr[v + 1]; ++k)
          vent.push_back((uint32_t)(v2fc[k] / 3) | (uint32_t)(v2fc[k] % 3) << 30);
      }
      vptr[H.n_own] = (int32_t)vent.size();
      if (vent.size() >= (size_t)kNone || nf >= (1 << 30))
        fail(IBM_ERR_UNSUPPORTED, "patch too large for 16-bit local indices; lower patch_size");
      for (size_t i = 0; i < vptr.size(); i += 2)
        T.fblob.push_back((uint32_t)vptr[i] | (i + 1 < vptr.size() ? (uint32_t)vptr[i + 1] << 16 : 0u));
      T.fblob.insert(T.fblob.end(), vent.begin(), vent.end());
      while (T.fblob.size() % 4) T.fblob.push_back(0u);
      Q.vf_words = (int32_t)T.fblob.size() - Q.blob_off - Q.blob_words;
      T.fpatch.push_back(Q);
      T.fface.insert(T.fface.end(), fo.begin(), fo.end());
    }
    T.max_loc = std::max(T.max_loc, H.n_loc);
    T.max_slot = std::max(T.max_slot, H.n_slot);
    T.max_own = std::max(T.max_own, H.n_own);
    T.patch.push_back(H);
  }
}

// Marker patches: the faces split by recursive coordinate bisection of their
// rest centroids into ceil(nf / kMT) compact parts of at most kMT faces (each
// split along the longest extent, at the quantile that keeps part counts
// balanced).  Writes the faces in patch order to `order` and the patch
// boundaries to `bounds` (size parts + 1).
void marker_patches(const int32_t* tri, int nf, const double* rest, std::vector<int32_t>& order,
                    std::vector<int32_t>& bounds, int PT) {
  std::vector<double> c(3 * (size_t)nf);
  for (int f = 0; f < nf; ++f)
    for (int d = 0; d < 3; ++d)
      c[3 * f + d] = (rest[3 * tri[3 * f] + d] + rest[3 * tri[3 * f + 1] + d] +
                      rest[3 * tri[3 * f + 2] + d]) / 3.0;
  order.resize(nf);
  for (int f = 0; f < nf; ++f) order[f] = f;
  bounds.assign(1, 0);
  struct Part {
    int lo, hi, parts;
  };
  std::vector<Part> stack{{0, nf, (nf + PT - 1) / PT}};
  std::vector<std::pair<int, int>> leaves;
  while (!stack.empty()) {
    Part p = stack.back();
    stack.pop_back();
    if (p.hi - p.lo <= PT) {
      leaves.push_back({p.lo, p.hi});
      continue;
    }
    p.parts = std::max(p.parts, (p.hi - p.lo + PT - 1) / PT);
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int k = p.lo; k < p.hi; ++k)
      for (int d = 0; d < 3; ++d) {
        lo[d] = std::min(lo[d], c[3 * order[k] + d]);
        hi[d] = std::max(hi[d], c[3 * order[k] + d]);
      }
    int ax = 0;
    for (int d = 1; d < 3; ++d)
      if (hi[d] - lo[d] > hi[ax] - lo[ax]) ax = d;
    const int p1 = p.parts / 2;
    const int mid = p.lo + (int)((long long)(p.hi - p.lo) * p1 / p.parts);
    std::stable_sort(order.begin() + p.lo, order.begin() + p.hi,
                     [&](int a, int b) { return c[3 * a + ax] < c[3 * b + ax]; });
    stack.push_back({mid, p.hi, p.parts - p1});
    stack.push_back({p.lo, mid, p1});
  }
  std::sort(leaves.begin(), leaves.end());
  for (auto& l : leaves) bounds.push_back(l.second);
}

uint64_t hash_mesh(const int32_t* t, int nf, int nv) {
  uint64_t h = 1469598103934665603ull ^ (uint64_t)nv;
  const unsigned char* p = reinterpret_cast<const unsigned char*>(t);
  for (size_t i = 0; i < (size_t)nf * 3 * sizeof(int32_t); ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

struct D3 {
  double x, y, z;
};
inline D3 dsub(D3 a, D3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline D3 dcross(D3 a, D3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
inline double ddot(D3 a, D3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline double dnorm(D3 a) { return std::sqrt(ddot(a, a)); }

template <class T>
T* upload(ibm_ctx* c, const std::vector<T>& h) {
  if (h.empty()) return nullptr;
  void* p = nullptr;
  check_cuda(cudaMalloc(&p, h.size() * sizeof(T)), "cudaMalloc");
  c->allocations.push_back(p);
  check_cuda(cudaMemcpy(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice), "upload");
  return static_cast<T*>(p);
}

template <class T>
T* zeros(ibm_ctx* c, size_t n) {
  if (n == 0) return nullptr;
  void* p = nullptr;
  check_cuda(cudaMalloc(&p, n * sizeof(T)), "cudaMalloc");
  c->allocations.push_back(p);
  check_cuda(cudaMemset(p, 0, n * sizeof(T)), "cudaMemset");
  return static_cast<T*>(p);
}

void free_all(ibm_ctx* c) {
  for (void* p : c->allocations) cudaFree(p);
  c->allocations.clear();
}

bool is_fin(double v) { return std::isfinite(v); }

// Within every full marker patch, store face t of the marker block's threads
// at position t, where thread t works on face W (t % 32) + t / 32 of the
// patch's spatial order (W warps): the warp's faces are spread over the patch
// (its simultaneous shared atomics of the spread rarely meet on a node) while
// its loads of the face records stay contiguous.
void interleave_full_patches(std::vector<int32_t>& mface, const std::vector<int32_t>& mbound,
                             int PT) {
  std::vector<int32_t> tmp(PT);
  for (size_t k = 0; k + 1 < mbound.size(); ++k) {
    if (mbound[k + 1] - mbound[k] != PT) continue;
    for (int t = 0; t < PT; ++t) tmp[t] = mface[mbound[k] + (PT / 32) * (t & 31) + (t >> 5)];
    std::copy(tmp.begin(), tmp.end(), mface.begin() + mbound[k]);
  }
}

// select body-sum buffer p (0 or 1) for the launches that follow
void use_parity(ibm_ctx* c, int p) {
  c->qpar = p;
  c->d.qsum = c->qsum_base + 2 * (size_t)c->B * p;
}

// power-of-two scale 2^e with ref * 2^e in [2^39, 2^40): the body's sum then
// has 2^22 of headroom in a 64-bit integer; false when 2^e is not a normal
// float
bool fixed_scale(double ref, float& s) {
  int ex = 0;
  std::frexp(ref, &ex);
  const int e = 40 - ex;
  if (!(ref > 0) || e < -120 || e > 120) return false;
  s = std::ldexp(1.0f, e);
  return true;
}

// fixed-point fields of a body record from A0, V0 and the constants
bool set_fixed_point(BodyDev& R) {
  if (!fixed_scale(R.A0, R.sA)) return false;
  R.qA0 = std::llrint(R.A0 * (double)R.sA);
  R.cA_unit = (float)((double)R.kA / ((double)R.sA * R.A0));
  if (R.closed) {
    if (!fixed_scale(R.V0, R.sV)) return false;
    R.qV0 = std::llrint(R.V0 * (double)R.sV);
    R.cV_unit = (float)((double)R.kv / ((double)R.sV * R.V0));
  } else {
    R.sV = 1.f;
    R.qV0 = 0;
    R.cV_unit = 0.f;
  }
  R.qlim = (float)(std::ldexp(1.0, 62) / (double)std::max(R.nf, 1));
  return true;
}

ibm_status set_err(ibm_ctx* c, ibm_status s, const std::string& m) {
  if (c) c->err = m;
  return s;
}

ibm_status cuda_status(ibm_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return IBM_OK;
  return set_err(c, IBM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Bound on |phi| of the closed-form MLS shape functions over every offset
// of the point from its nearest node: |phi| <= prod_d (max_s a_s + max_s |b_s|)
// (phi = a_x a_y a_z - b_x a_y a_z - a_x b_y a_z - a_x a_y b_z), the factors
// taken over a fine sweep of the fractional offset, with a margin.
double phi_bound_of(double kappa) {
  double best = 0.0;
  for (int k = 0; k <= 20000; ++k) {
    const double tp = -0.5 + k / 20000.0;
    const double rm = std::exp(-kappa * (1 + 2 * tp)), rp = std::exp(-kappa * (1 - 2 * tp));
    const double S = 1 + rm + rp;
    const double a[3] = {rm / S, 1 / S, rp / S}, d[3] = {-1 - tp, -tp, 1 - tp};
    const double mu = a[0] * d[0] + a[1] * d[1] + a[2] * d[2];
    double s2 = 0.0;
    for (int j = 0; j < 3; ++j) s2 += a[j] * (d[j] - mu) * (d[j] - mu);
    double amax = 0.0, bmax = 0.0;
    for (int j = 0; j < 3; ++j) {
      amax = std::max(amax, a[j]);
      bmax = std::max(bmax, std::fabs(a[j] * mu * (d[j] - mu) / s2));
    }
    best = std::max(best, amax + bmax);
  }
  return 1.05 * best * best * best;
}

// the step's marker kernel: body sums, interpolation, traction and spread
// with the previous footprint cleared (clear) or accumulated
cudaError_t launch_step_marker(ibm_ctx* c, const float* x, const float* v, const float* u,
                               const float* vv, const float* w, const float* p,
                               const float* accel, float* fx, float* fy, float* fz, bool clear,
                               bool after_clear) {
  // after_clear: the footprint clear is the launch just before this one on
  // the same stream (nothing between them), so the marker kernel may overlap it
  return launch_mls(c, x, v, u, vv, w, p, accel, nullptr, nullptr, nullptr, c->d.fext, fx, fy, fz,
                    true, true, true, true, clear, after_clear && !c->timing);
}

void make_consts(ibm_ctx* c) {
  const ibm_params& p = c->prm;
  ibm::Grid& g = c->grid;
  double h[3];
  for (int d = 0; d < 3; ++d) {
    g.n[d] = c->gdesc.n[d];
    h[d] = c->gdesc.L[d] / c->gdesc.n[d];
    g.h[d] = (float)h[d];
    g.invh[d] = (float)(1.0 / h[d]);
  }
  const double alpha = p.alpha > 0 ? p.alpha : 0.3;
  c->sc.dt = (float)p.dt;
  c->sc.inv_dt = (float)(1.0 / p.dt);
  c->sc.mu = (float)p.mu;
  c->sc.probe_h = (float)(p.probe_h > 0 ? p.probe_h : (h[0] + h[1] + h[2]) / 3.0);
  c->sc.kappa = (float)(1.0 / ((1.5 * alpha) * (1.5 * alpha)));
  c->sc.cl_scale = (float)(((h[0] + h[1] + h[2]) / 3.0) / (h[0] * h[1] * h[2]));
  c->sc.forward_euler = p.forward_euler ? 1 : 0;
  const char* st = std::getenv("IBM_TEST_STARVE_TX");
  c->sc.starve_tx = st ? std::max(0, std::min(std::atoi(st), 1024)) : 0;
  c->phi_bound = (float)phi_bound_of(c->sc.kappa);
}

}  // namespace

void ibm::set_global_error(const std::string& msg) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_err = msg;
}

// ---------------------------------------------------------------------------
// entry points
// ---------------------------------------------------------------------------

extern "C" ibm_status ibm_create_bodies(ibm_ctx** out, const ibm_body_desc* bodies,
                                        int32_t n_bodies, const ibm_grid_desc* grid,
                                        const ibm_params* params, int32_t device) {
  if (out) *out = nullptr;
  ibm_ctx* c = nullptr;
  try {
    if (!out || !bodies || !grid || !params || n_bodies <= 0)
      fail(IBM_ERR_INVALID_ARG, "null argument or n_bodies <= 0");
    int ndev = 0;
    cudaError_t ce = cudaGetDeviceCount(&ndev);
    if (ce != cudaSuccess || ndev == 0)
      fail(IBM_ERR_CUDA, std::string("no usable CUDA device: ") + cudaGetErrorString(ce));
    if (device < 0 || device >= ndev) fail(IBM_ERR_INVALID_ARG, "device index out of range");
    check_cuda(cudaSetDevice(device), "cudaSetDevice");
    // grid and parameters
    long long nodes = 1;
    for (int d = 0; d < 3; ++d) {
      if (grid->n[d] < 4 || grid->n[d] > (1 << 16))
        fail(IBM_ERR_INVALID_ARG, "grid n must be in [4, 65536] per direction");
      if (!is_fin(grid->L[d]) || grid->L[d] <= 0) fail(IBM_ERR_INVALID_ARG, "grid L must be > 0");
      nodes *= grid->n[d];
    }
    if (nodes >= (1ll << 31)) fail(IBM_ERR_UNSUPPORTED, "grid has 2^31 or more nodes");
    const ibm_params& p = *params;
    if (!is_fin(p.dt) || p.dt <= 0) fail(IBM_ERR_INVALID_ARG, "dt must be finite and > 0");
    if (!is_fin(p.mu) || p.mu < 0) fail(IBM_ERR_INVALID_ARG, "mu must be finite and >= 0");
    if (!is_fin(p.alpha) || p.alpha < 0) fail(IBM_ERR_INVALID_ARG, "alpha must be >= 0");
    if (!is_fin(p.probe_h)) fail(IBM_ERR_INVALID_ARG, "probe_h must be finite");
    const int P = p.patch_size > 0 ? p.patch_size : 128;
    static_assert(kMirrorChunk >= 2048, "a patch's own run meets at most two mirror chunks");
    if (P < 32 || P > 2048) fail(IBM_ERR_INVALID_ARG, "patch_size must be in [32, 2048]");
    if (p.spread_variant < 0 || p.spread_variant > 2)
      fail(IBM_ERR_INVALID_ARG, "spread_variant must be 0, 1 or 2");
    if (p.marker_patch != 0 && p.marker_patch != 128 && p.marker_patch != 256)
      fail(IBM_ERR_INVALID_ARG, "marker_patch must be 0, 128 or 256");

    c = new ibm_ctx();
    c->device = device;
    c->prm = p;
    c->prm.patch_size = P;
    c->spread_variant = p.spread_variant == 0 ? 1 : p.spread_variant;
    c->prm.spread_variant = c->spread_variant;
    c->marker_patch = p.marker_patch == 0 ? kMT : p.marker_patch;
    c->prm.marker_patch = c->marker_patch;
    c->gdesc = *grid;
    make_consts(c);
    double h[3];
    for (int d = 0; d < 3; ++d) h[d] = grid->L[d] / grid->n[d];

    // topologies, shared between bodies with identical faces
    std::vector<HostTopo> topos;
    std::unordered_map<uint64_t, std::vector<int>> by_hash;
    std::vector<int> body_topo(n_bodies);
    for (int b = 0; b < n_bodies; ++b) {
      const ibm_body_desc& B = bodies[b];
      if (B.n_vert < 3 || B.n_face < 1 || !B.rest || !B.tri)
        fail(IBM_ERR_INVALID_ARG, "body " + std::to_string(b) + ": needs >= 3 vertices, >= 1 face");
      const uint64_t hsh = hash_mesh(B.tri, B.n_face, B.n_vert);
      int found = -1;
      for (int t : by_hash[hsh]) {
        const HostTopo& T = topos[t];
        if (T.nv == B.n_vert && T.nf == B.n_face &&
            std::memcmp(T.tri.data(), B.tri, sizeof(int32_t) * 3 * (size_t)B.n_face) == 0) {
          found = t;
          break;
        }
      }
      if (found < 0) {
        topos.emplace_back();
        try {
          build_topology(topos.back(), B.tri, B.n_vert, B.n_face, P);
          marker_patches(B.tri, B.n_face, B.rest, topos.back().mface, topos.back().mbound,
                         c->marker_patch);
          interleave_full_patches(topos.back().mface, topos.back().mbound, c->marker_patch);

        } catch (Failure& f) {
          f.msg = "body " + std::to_string(b) + ": " + f.msg;
          throw;
        }
        found = (int)topos.size() - 1;
        by_hash[hsh].push_back(found);
      }
      body_topo[b] = found;
      if (B.closed && topos[found].has_boundary)
        fail(IBM_ERR_MESH, "body " + std::to_string(b) + " is marked closed but has boundary edges");
    }
    // body records and rest state (float64)
    long long V = 0, F = 0, E = 0;
    for (int b = 0; b < n_bodies; ++b) {
      V += bodies[b].n_vert;
      F += bodies[b].n_face;
      E += topos[body_topo[b]].ne;
    }
    if (V >= (1ll << 31) / 3 || F >= (1ll << 31) / 3 || E >= (1ll << 31))
      fail(IBM_ERR_UNSUPPORTED, "too many vertices/faces for 32-bit indexing");
    c->V = V;
    c->F = F;
    c->E = E;
    c->B = n_bodies;
    c->n_topo = (int)topos.size();
    std::vector<float> rest(3 * V), l0(E), A0f(F);
    std::vector<float2> cs0(E);
    // per-element multipliers of k_s (edges), k_b (hinges), k_a (faces);
    // filled only when some body has a non-uniform spring model or materials
    std::vector<float> kse, kbe, kaf;
    bool any_varied = false;
    for (int b = 0; b < n_bodies; ++b)
      any_varied = any_varied || bodies[b].spring_model != 0 || bodies[b].face_material != nullptr;
    if (any_varied) {
      kse.assign(E, 1.f);
      kbe.assign(E, 1.f);
      kaf.assign(F, 1.f);
    }
    std::vector<uint8_t> clamp(V, 0);
    std::vector<int4> chunks;
    std::vector<int2> work;
    std::vector<float> frest;        // force-kernel rest data per work item, patch order
    std::vector<int64_t> wrest;
    size_t force_smem = 0, adjoint_smem = 0;
    c->h_body.resize(n_bodies);
    long long vo = 0, fo = 0, eo = 0;
    for (int b = 0; b < n_bodies; ++b) {
      const ibm_body_desc& Bd = bodies[b];
      const HostTopo& T = topos[body_topo[b]];
      const std::string tag = "body " + std::to_string(b) + ": ";
      const double kk[6] = {Bd.ks, Bd.kb, Bd.ka, Bd.kA, Bd.kv, Bd.mass};
      for (double k : kk)
        if (!is_fin(k)) fail(IBM_ERR_INVALID_ARG, tag + "non-finite elastic constant or mass");
      if (Bd.mass <= 0) fail(IBM_ERR_INVALID_ARG, tag + "mass must be > 0");
      for (int d = 0; d < 3; ++d)
        if (!is_fin(Bd.origin[d])) fail(IBM_ERR_INVALID_ARG, tag + "non-finite origin");
      std::vector<D3> x(Bd.n_vert);
      for (int v = 0; v < Bd.n_vert; ++v) {
        x[v] = {Bd.rest[3 * v] - Bd.origin[0], Bd.rest[3 * v + 1] - Bd.origin[1],
                Bd.rest[3 * v + 2] - Bd.origin[2]};
        if (!is_fin(x[v].x) || !is_fin(x[v].y) || !is_fin(x[v].z))
          fail(IBM_ERR_INVALID_ARG, tag + "non-finite rest position");
        rest[vo + v] = (float)x[v].x;
        rest[V + vo + v] = (float)x[v].y;
        rest[2 * V + vo + v] = (float)x[v].z;
        if (Bd.clamped) clamp[vo + v] = Bd.clamped[v] ? 1 : 0;
      }
      for (int e = 0; e < T.ne; ++e) {
        const int4 Ed = T.edge[e];
        const D3 ev = dsub(x[Ed.y], x[Ed.x]);
        const double l = dnorm(ev);
        if (!(l > 0)) fail(IBM_ERR_MESH, tag + "zero-length rest edge");
        l0[eo + e] = (float)l;
        float2 cs = make_float2(1.f, 0.f);
        if (Ed.w >= 0 && !p.theta0_zero) {
          const D3 N1 = dcross(ev, dsub(x[Ed.z], x[Ed.x]));
          const D3 N2 = dcross(dsub(x[Ed.w], x[Ed.y]), ev);
          const double n1 = dnorm(N1), n2 = dnorm(N2);
          const D3 a = {N1.x / n1, N1.y / n1, N1.z / n1}, bb = {N2.x / n2, N2.y / n2, N2.z / n2};
          const double ct = ddot(a, bb);
          const double st = ddot(dcross(a, bb), ev) / l;
          cs = make_float2((float)ct, (float)st);
        }
        cs0[eo + e] = cs;
      }
      double A0 = 0.0, V0 = 0.0;
      std::vector<double> a0(T.nf);
      for (int f = 0; f < T.nf; ++f) {
        const D3 xa = x[T.tri[3 * f]], xb = x[T.tri[3 * f + 1]], xc = x[T.tri[3 * f + 2]];
        const double a = 0.5 * dnorm(dcross(dsub(xb, xa), dsub(xc, xa)));
        if (!(a > 0)) fail(IBM_ERR_MESH, tag + "degenerate (zero-area) rest face");
        A0f[fo + f] = (float)a;
        a0[f] = a;
        A0 += a;
        V0 += ddot(xa, dcross(xb, xc)) / 6.0;
      }
      const bool varied = Bd.spring_model != 0 || Bd.face_material != nullptr;
      if (Bd.spring_model != 0 && Bd.spring_model != 1)
        fail(IBM_ERR_INVALID_ARG, tag + "spring_model must be 0 (uniform) or 1 (van Gelder)");
      if (varied) {
        // face multipliers (m_s, m_b, m_a); an edge takes the mean of its
        // faces' m_s, or under van Gelder sum_T m_s(T) A_T / l^2; a hinge the
        // mean of its two faces' m_b; a face its own m_a
        auto mat = [&](int f, int j) -> double {
          return Bd.face_material ? (double)Bd.face_material[3 * f + j] : 1.0;
        };
        if (Bd.face_material)
          for (int f = 0; f < T.nf; ++f)
            for (int j = 0; j < 3; ++j)
              if (!(mat(f, j) >= 0.0) || !is_fin(mat(f, j)))
                fail(IBM_ERR_INVALID_ARG, tag + "face_material must be finite and >= 0");
        for (int e = 0; e < T.ne; ++e) {
          const int2 ef = T.eface[e];
          const int4 Ed = T.edge[e];
          const double l = dnorm(dsub(x[Ed.y], x[Ed.x]));
          double ms;
          if (Bd.spring_model == 1) {
            ms = mat(ef.x, 0) * a0[ef.x] + (ef.y >= 0 ? mat(ef.y, 0) * a0[ef.y] : 0.0);
            ms /= l * l;
          } else {
            ms = ef.y >= 0 ? 0.5 * (mat(ef.x, 0) + mat(ef.y, 0)) : mat(ef.x, 0);
          }
          kse[eo + e] = (float)ms;
          kbe[eo + e] = ef.y >= 0 ? (float)(0.5 * (mat(ef.x, 1) + mat(ef.y, 1))) : 0.f;
        }
        for (int f = 0; f < T.nf; ++f) kaf[fo + f] = (float)mat(f, 2);
      }
      if (Bd.closed && !(V0 > 0))
        fail(IBM_ERR_MESH, tag + "closed body with non-positive rest volume (faces oriented inward?)");
      BodyDev& R = c->h_body[b];
      std::memset(&R, 0, sizeof(R));
      R.v_off = (int32_t)vo;
      R.f_off = (int32_t)fo;
      R.e_off = (int32_t)eo;
      R.topo = body_topo[b];
      R.nv = Bd.n_vert;
      R.nf = Bd.n_face;
      R.ne = T.ne;
      R.closed = Bd.closed ? 1 : 0;
      R.varied = varied ? 1 : 0;
      for (int d = 0; d < 3; ++d) {
        const double o = Bd.origin[d] / h[d];
        const double Gd = std::floor(o);
        R.frac[d] = (float)(o - Gd);
        R.fracd[d] = o - Gd;
        long long Gi = (long long)Gd % grid->n[d];
        if (Gi < 0) Gi += grid->n[d];
        R.G[d] = (int32_t)Gi;
      }
      R.ks = (float)Bd.ks;
      R.kb = (float)Bd.kb;
      R.ka = (float)Bd.ka;
      R.kA = (float)Bd.kA;
      R.kv = Bd.closed ? (float)Bd.kv : 0.f;
      R.inv_mass = (float)(1.0 / Bd.mass);
      R.A0 = A0;
      R.V0 = Bd.closed ? V0 : 1.0;
      if (!set_fixed_point(R))
        fail(IBM_ERR_MESH, tag + "rest area or volume outside the supported range");
      R.chunk_off = (int32_t)chunks.size();
      const int nch = (int)T.mbound.size() - 1;
      R.n_chunk = nch;
      for (int k = 0; k < nch; ++k)
        chunks.push_back(make_int4(b, T.mbound[k], T.mbound[k + 1] - T.mbound[k], k));
      R.work_off = (int32_t)work.size();
      for (int q = 0; q < (int)T.patch.size(); ++q) {
        work.push_back(make_int2(b, q));
        const PatchHdr& H = T.patch[q];
        const int pe = pad4(H.n_edge), pf = pad4(H.n_face);
        const size_t r0 = frest.size();
        wrest.push_back((int64_t)r0);
        frest.resize(r0 + frest_words(H.n_edge, H.n_face, varied), 0.f);
        for (int i = 0; i < H.n_edge; ++i) {
          const long long ge = eo + (T.pedge[H.edge_off + i].eid & 0x7fffffff);
          frest[r0 + i] = l0[ge];
          frest[r0 + pe + i] = cs0[ge].x;
          frest[r0 + 2 * pe + i] = cs0[ge].y;
          if (varied) {
            frest[r0 + 3 * pe + pf + i] = kse[ge];
            frest[r0 + 4 * pe + pf + i] = kbe[ge];
          }
        }
        for (int i = 0; i < H.n_face; ++i) {
          const long long gf = fo + T.fface[H.face_off + i];
          frest[r0 + 3 * pe + i] = A0f[gf];
          if (varied) frest[r0 + 5 * pe + pf + i] = kaf[gf];
        }
        // shared memory of the block: blob, rest data, positions, slots
        const FPatch& Q = T.fpatch[q];
        force_smem = std::max(force_smem,
                              sizeof(float) * ((size_t)Q.blob_words + frest_words(H.n_edge, H.n_face, varied) +
                                               3 * (size_t)pad4(H.n_loc) + 3 * (size_t)pad4(Q.n_slot)));
        // the adjoint: blob with its tail, rest data, positions and
        // tangents, slots
        adjoint_smem = std::max(
            adjoint_smem, sizeof(float) * ((size_t)Q.blob_words + Q.vf_words +
                                           frest_words(H.n_edge, H.n_face, varied) +
                                           6 * (size_t)pad4(H.n_loc) + 3 * (size_t)pad4(Q.n_slot)));
      }
      vo += Bd.n_vert;
      fo += Bd.n_face;
      eo += T.ne;
    }
    c->n_chunks = (int32_t)chunks.size();
    c->n_work = (int32_t)work.size();

    // concatenate the topology tables
    std::vector<TopoDev> td(topos.size());
    std::vector<int32_t> tri_all, v2f_ptr_all, v2f_idx_all, loc_all, csr_all, mface_all;
    std::vector<int4> mtri_all;
    std::vector<int4> edge_all;
    std::vector<PatchHdr> patch_all;
    std::vector<PEdge> pedge_all;
    std::vector<PFace> pface_all;
    std::vector<uint16_t> slot_all;
    std::vector<uint32_t> fblob_all;
    std::vector<FPatch> fpatch_all;
    int max_loc = 0, max_slot = 0, max_own = 0;
    for (size_t t = 0; t < topos.size(); ++t) {
      const HostTopo& T = topos[t];
      TopoDev& D = td[t];
      std::memset(&D, 0, sizeof(D));
      D.nv = T.nv;
      D.nf = T.nf;
      D.ne = T.ne;
      D.n_patch = (int32_t)T.patch.size();
      D.tri_off = (int32_t)tri_all.size();
      tri_all.insert(tri_all.end(), T.tri.begin(), T.tri.end());
      D.edge_off = (int32_t)edge_all.size();
      edge_all.insert(edge_all.end(), T.edge.begin(), T.edge.end());
      D.v2f_ptr_off = (int32_t)v2f_ptr_all.size();
      v2f_ptr_all.insert(v2f_ptr_all.end(), T.v2f_ptr.begin(), T.v2f_ptr.end());
      D.v2f_idx_off = (int32_t)v2f_idx_all.size();
      v2f_idx_all.insert(v2f_idx_all.end(), T.v2f_idx.begin(), T.v2f_idx.end());
      D.mface_off = (int32_t)mface_all.size();
      mface_all.insert(mface_all.end(), T.mface.begin(), T.mface.end());
      for (const int32_t f : T.mface)
        mtri_all.push_back(make_int4(T.tri[3 * f], T.tri[3 * f + 1], T.tri[3 * f + 2], f));

      D.patch_off = (int32_t)patch_all.size();
      const int32_t lo = (int32_t)loc_all.size(), eo2 = (int32_t)pedge_all.size(),
                    fo2 = (int32_t)pface_all.size(), co = (int32_t)csr_all.size(),
                    so = (int32_t)slot_all.size();
      for (PatchHdr H : T.patch) {
        H.loc_off += lo;
        H.edge_off += eo2;
        H.face_off += fo2;
        H.csr_off += co;
        H.slot_off += so;
        patch_all.push_back(H);
      }
      loc_all.insert(loc_all.end(), T.loc_vert.begin(), T.loc_vert.end());
      pedge_all.insert(pedge_all.end(), T.pedge.begin(), T.pedge.end());
      pface_all.insert(pface_all.end(), T.pface.begin(), T.pface.end());
      csr_all.insert(csr_all.end(), T.csr_ptr.begin(), T.csr_ptr.end());
      slot_all.insert(slot_all.end(), T.csr_slot.begin(), T.csr_slot.end());
      const int32_t bo = (int32_t)fblob_all.size();
      for (FPatch Q : T.fpatch) {
        Q.blob_off += bo;
        fpatch_all.push_back(Q);
      }
      fblob_all.insert(fblob_all.end(), T.fblob.begin(), T.fblob.end());
      max_loc = std::max(max_loc, T.max_loc);
      max_slot = std::max(max_slot, T.max_slot);
      max_own = std::max(max_own, T.max_own);
    }
    (void)max_slot;
    c->force_smem = force_smem;
    if (c->force_smem > 227 * 1024)
      fail(IBM_ERR_UNSUPPORTED, "force-kernel shared memory above 227 KB; lower patch_size");
    c->adjoint_smem = adjoint_smem;
    c->max_own = max_own;
    if (c->adjoint_smem > 227 * 1024)
      fail(IBM_ERR_UNSUPPORTED, "force-kernel shared memory above 227 KB; lower patch_size");
    check_cuda(set_force_smem_limit(c->force_smem), "cudaFuncSetAttribute");
    check_cuda(set_adjoint_smem_limit(c->adjoint_smem), "cudaFuncSetAttribute");
    check_cuda(set_marker_smem_limit(), "cudaFuncSetAttribute");
    c->vec4 = (grid->n[0] % 4 == 0) ? 1 : 0;

    DeviceTables& d = c->d;
    d.body = upload(c, c->h_body);
    d.topo = upload(c, td);
    d.tri = upload(c, tri_all);
    d.edge = upload(c, edge_all);
    d.v2f_ptr = upload(c, v2f_ptr_all);
    d.v2f_idx = upload(c, v2f_idx_all);
    d.patch = upload(c, patch_all);
    d.loc_vert = upload(c, loc_all);
    d.pedge = upload(c, pedge_all);
    d.pface = upload(c, pface_all);
    d.csr_ptr = upload(c, csr_all);
    d.csr_slot = upload(c, slot_all);
    d.fblob = upload(c, fblob_all);
    d.fpatch = upload(c, fpatch_all);
    d.frest = upload(c, frest);
    d.wrest = upload(c, wrest);
    d.l0 = upload(c, l0);
    d.cs0 = upload(c, cs0);
    d.A0f = upload(c, A0f);
    if (any_varied) {
      d.kse = upload(c, kse);
      d.kbe = upload(c, kbe);
      d.kaf = upload(c, kaf);
    }
    d.clamp = upload(c, clamp);
    d.rest = upload(c, rest);
    d.chunks = upload(c, chunks);
    d.work = upload(c, work);
    c->qsum_base = zeros<unsigned long long>(c, 4 * (size_t)n_bodies);
    d.qsum = c->qsum_base;
    d.meas = zeros<double>(c, 2 * (size_t)n_bodies);
    d.fext = zeros<float>(c, 3 * (size_t)F);
    d.err = zeros<int32_t>(c, 1);
    d.coef = zeros<float2>(c, (size_t)n_bodies);
    d.boxes = zeros<int4>(c, 2 * (size_t)c->n_chunks);
    d.rowmap = zeros<int2>(c, (size_t)kMaxRows * c->n_chunks);
    d.mface = upload(c, mface_all);
    d.mtri = upload(c, mtri_all);
    d.stats = zeros<int32_t>(c, 4);
    d.partial2 = zeros<double>(c, 2 * (size_t)c->n_chunks);
    d.counter2 = zeros<int32_t>(c, (size_t)n_bodies);
    d.dmeas = zeros<double>(c, 2 * (size_t)n_bodies);
    d.gxe = zeros<float>(c, 9 * (size_t)F);
    d.wpart = zeros<double>(c, 3 * (size_t)c->n_work);
    d.wcounter = zeros<int32_t>(c, (size_t)n_bodies);
    d.tpart = zeros<double>(c, 10 * (size_t)c->n_chunks);
    d.taylor = zeros<double>(c, 24 * (size_t)n_bodies);
    d.tgrad = zeros<double>(c, 10 * (size_t)n_bodies);
    if (c->spread_variant == 2) {
      // tile tables of the tile-owned spread; the marker list holds at most
      // (tiles per direction a 4-node support can reach)^3 entries per marker:
      // 2 per direction, 3 where a partial last tile has fewer than 3 nodes
      TileDev& t = c->td;
      const int TT[3] = {kTX, kTY, kTZ};
      long long per = 1;
      for (int k = 0; k < 3; ++k) {
        t.nt[k] = (grid->n[k] + TT[k] - 1) / TT[k];
        const int rem = grid->n[k] % TT[k];
        per *= t.nt[k] == 1 ? 1 : ((rem == 1 || rem == 2) ? 3 : 2);
      }
      t.n_tiles = t.nt[0] * t.nt[1] * t.nt[2];
      c->max_pairs = per * (long long)F;
      if (c->max_pairs >= (1ll << 31))
        fail(IBM_ERR_UNSUPPORTED, "tile-owned spread: more than 2^31 marker-tile pairs possible");
      t.count = zeros<int32_t>(c, t.n_tiles);
      t.off = zeros<int32_t>(c, t.n_tiles);
      t.cur = zeros<int32_t>(c, t.n_tiles);
      t.epoch = zeros<int32_t>(c, t.n_tiles);
      check_cuda(cudaMemset(t.epoch, 0xff, sizeof(int32_t) * t.n_tiles), "cudaMemset");
      t.mask = zeros<uint32_t>(c, 12 * (size_t)t.n_tiles);
      t.tmax = zeros<uint32_t>(c, 4 * (size_t)t.n_tiles);
      t.active[0] = zeros<int32_t>(c, t.n_tiles);
      t.state = zeros<int32_t>(c, 8);
      t.mlist = zeros<int32_t>(c, (size_t)std::max<long long>(c->max_pairs, 1));
      t.rec = zeros<float4>(c, 2 * (size_t)F);
      int per_sm = 0, n_sm = 0;
      check_cuda(tile_spread_occupancy(&per_sm), "occupancy");
      check_cuda(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device), "attr");
      c->tile_grid = std::max(1, per_sm) * std::max(1, n_sm);
      check_cuda(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking), "cudaStreamCreate");
      check_cuda(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming), "cudaEventCreate");
      check_cuda(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming), "cudaEventCreate");
    }
    check_cuda(cudaDeviceSynchronize(), "create");
    *out = c;
    return IBM_OK;
  } catch (Failure& f) {
    if (c) {
      free_all(c);
      delete c;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    g_err = f.msg;
    return f.s;
  } catch (std::exception& e) {
    if (c) {
      free_all(c);
      delete c;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    g_err = std::string("host error: ") + e.what();
    return IBM_ERR_OOM;
  }
}

extern "C" void ibm_destroy(ibm_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (auto& ev : c->ev)
    if (ev) cudaEventDestroy(ev);
  if (c->side) {
    cudaStreamSynchronize(c->side);
    cudaStreamDestroy(c->side);
  }
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->hcopy) {
    cudaStreamSynchronize(c->hcopy);
    cudaStreamDestroy(c->hcopy);
  }
  if (c->ev_hfork) cudaEventDestroy(c->ev_hfork);
  if (c->ev_hcopy) cudaEventDestroy(c->ev_hcopy);
  free_all(c);
  delete c;
}

extern "C" const char* ibm_last_error(const ibm_ctx* c) {
  if (c) return c->err.c_str();
  std::lock_guard<std::mutex> lk(g_mu);
  return g_err.c_str();
}

extern "C" ibm_status ibm_set_stream(ibm_ctx* c, void* stream) {
  if (!c) return IBM_ERR_INVALID_ARG;
  c->stream = static_cast<cudaStream_t>(stream);
  return IBM_OK;
}

extern "C" ibm_status ibm_get_sizes(const ibm_ctx* c, int64_t* out) {
  if (!c || !out) return IBM_ERR_INVALID_ARG;
  out[0] = c->V;
  out[1] = c->F;
  out[2] = c->E;
  out[3] = c->B;
  out[4] = c->n_topo;
  out[5] = c->n_work;
  return IBM_OK;
}

extern "C" ibm_status ibm_get_params(const ibm_ctx* c, ibm_params* out) {
  if (!c || !out) return IBM_ERR_INVALID_ARG;
  *out = c->prm;
  if (!(out->alpha > 0)) out->alpha = 0.3;
  out->probe_h = c->sc.probe_h;
  return IBM_OK;
}

extern "C" ibm_status ibm_get_offsets(const ibm_ctx* c, int64_t* out) {
  if (!c || !out) return IBM_ERR_INVALID_ARG;
  for (size_t b = 0; b < c->h_body.size(); ++b) {
    out[3 * b] = c->h_body[b].v_off;
    out[3 * b + 1] = c->h_body[b].f_off;
    out[3 * b + 2] = c->h_body[b].e_off;
  }
  return IBM_OK;
}

extern "C" ibm_status ibm_init_state(ibm_ctx* c, float* x, float* v) {
  if (!c || !x || !v) return set_err(c, IBM_ERR_INVALID_ARG, "null argument");
  cudaSetDevice(c->device);
  cudaError_t e = cudaMemcpyAsync(x, c->d.rest, sizeof(float) * 3 * c->V,
                                  cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(v, 0, sizeof(float) * 3 * c->V, c->stream);
  return cuda_status(c, e, "ibm_init_state");
}

extern "C" ibm_status ibm_set_body_constants(ibm_ctx* c, const double* k) {
  if (!c || !k) return set_err(c, IBM_ERR_INVALID_ARG, "null argument");
  for (int64_t b = 0; b < c->B; ++b) {
    for (int j = 0; j < 6; ++j)
      if (!is_fin(k[6 * b + j])) return set_err(c, IBM_ERR_INVALID_ARG, "non-finite constant");
    if (k[6 * b + 5] <= 0) return set_err(c, IBM_ERR_INVALID_ARG, "mass must be > 0");
    BodyDev& R = c->h_body[b];
    R.ks = (float)k[6 * b];
    R.kb = (float)k[6 * b + 1];
    R.ka = (float)k[6 * b + 2];
    R.kA = (float)k[6 * b + 3];
    R.kv = R.closed ? (float)k[6 * b + 4] : 0.f;
    R.inv_mass = (float)(1.0 / k[6 * b + 5]);
    set_fixed_point(R);
  }
  cudaSetDevice(c->device);
  // synchronous with respect to the host buffer (pageable source)
  cudaError_t e = cudaMemcpyAsync(c->d.body, c->h_body.data(), sizeof(BodyDev) * c->B,
                                  cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return cuda_status(c, e, "ibm_set_body_constants");
}

extern "C" ibm_status ibm_body_measures(ibm_ctx* c, const float* x, double* out) {
  if (!c || !x || !out) return set_err(c, IBM_ERR_INVALID_ARG, "null argument");
  cudaSetDevice(c->device);
  cudaError_t e = zero_body_sums(c);
  if (e == cudaSuccess)
    e = launch_mls(c, x, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                   nullptr, nullptr, nullptr, nullptr, nullptr, true, false, false, false, false);
  if (e == cudaSuccess) e = launch_measure_finalize(c);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, c->d.meas, sizeof(double) * 2 * c->B, cudaMemcpyDeviceToDevice,
                        c->stream);
  return cuda_status(c, e, "ibm_body_measures");
}

extern "C" ibm_status ibm_compute_forces(ibm_ctx* c, const float* x, float* F_int,
                                         double* energy) {
  if (!c || !x || !F_int) return set_err(c, IBM_ERR_INVALID_ARG, "null argument");
  cudaSetDevice(c->device);
  cudaError_t e = zero_body_sums(c);
  if (e == cudaSuccess)
    e = launch_mls(c, x, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                   nullptr, nullptr, nullptr, nullptr, nullptr, true, false, false, false, false);
  if (e == cudaSuccess && energy) e = launch_measure_finalize(c);
  if (e == cudaSuccess && energy)
    e = cudaMemsetAsync(energy, 0, sizeof(double) * 5 * c->B, c->stream);
  if (e == cudaSuccess)
    e = launch_force(c, x, nullptr, nullptr, F_int, nullptr, nullptr, energy, false);
  return cuda_status(c, e, "ibm_compute_forces");
}

extern "C" ibm_status ibm_interpolate(ibm_ctx* c, const float* x, const float* v, const float* u,
                                      const float* vv, const float* w, const float* p,
                                      const float* accel, float* U, float* Fm, float* Fext) {
  if (!c || !x || !u || !vv || !w) return set_err(c, IBM_ERR_INVALID_ARG, "null argument");
  if (Fm && !v) return set_err(c, IBM_ERR_INVALID_ARG, "F_marker needs the vertex velocities");
  const bool interp = U || Fm;
  const bool probe = Fext != nullptr;
  if (!interp && !probe) return IBM_OK;
  cudaSetDevice(c->device);
  cudaError_t e = launch_mls(c, x, v, u, vv, w, p, accel, U, Fm, nullptr, Fext, nullptr, nullptr,
                             nullptr, false, interp, probe, false, false);
  return cuda_status(c, e, "ibm_interpolate");
}

extern "C" ibm_status ibm_interpolate_fp64(ibm_ctx* c, const float* x, const float* v,
                                           const float* u, const float* vv, const float* w,
                                           float* U, float* Fm, float* Fext) {
  if (!c || !x || !u || !vv || !w) return set_err(c, IBM_ERR_INVALID_ARG, "null argument");
  if (Fm && !v) return set_err(c, IBM_ERR_INVALID_ARG, "F_marker needs the vertex velocities");
  if (!U && !Fm && !Fext) return IBM_OK;
  cudaSetDevice(c->device);
  return cuda_status(c, launch_interp64(c, x, v, u, vv, w, U, Fm, Fext), "ibm_interpolate_fp64");
}

extern "C" ibm_status ibm_advance(ibm_ctx* c, const float* x, const float* v, const float* F_int,
                                  const float* F_ext, float* x_out, float* v_out) {
  if (!c || !x || !v || !F_int || !F_ext || !x_out || !v_out)
    return set_err(c, IBM_ERR_INVALID_ARG, "null argument");
  cudaSetDevice(c->device);
  return cuda_status(c, launch_advance(c, x, v, F_int, F_ext, x_out, v_out), "ibm_advance");
}

extern "C" ibm_status ibm_spread(ibm_ctx* c, const float* x, const float* Fm, float* fx, float* fy,
                                 float* fz) {
  if (!c || !x || !Fm || !fx || !fy || !fz) return set_err(c, IBM_ERR_INVALID_ARG, "null argument");
  cudaSetDevice(c->device);
  cudaError_t e = cudaSuccess;
  if (c->spread_variant == 2) {
    e = launch_tile_begin(c, true, false);
    if (e == cudaSuccess)
      e = launch_mls_records(c, x, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, Fm,
                             nullptr, false, false, true);
    if (e == cudaSuccess) e = launch_tile_spread(c, fx, fy, fz, true);
  } else {
    e = launch_mls(c, x, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, Fm,
                   nullptr, fx, fy, fz, false, false, false, true, false);
  }
  return cuda_status(c, e, "ibm_spread");
}

namespace {

// The launches of one ibm_step on the context's stream.  before_marker
// (optional): an event the marker kernel must wait for (inputs copied in on
// another stream); the footprint clear or set-up runs before that wait.
cudaError_t step_launches(ibm_ctx* c, const float* x, const float* v, const float* u,
                          const float* vv, const float* w, const float* p, const float* accel,
                          float* x_out, float* v_out, float* fx, float* fy, float* fz,
                          uint32_t flags, cudaEvent_t before_marker,
                          const Mirror* mirror = nullptr) {
  const bool clear = (flags & IBM_STEP_CLEAR_PREV) != 0;
  use_parity(c, c->qpar ^ 1);
  cudaError_t e = cudaSuccess;
  auto mark = [&](int k) {
    if (c->timing && e == cudaSuccess) e = cudaEventRecord(c->ev[k], c->stream);
  };
  mark(0);
  if (c->spread_variant == 2) {
    // set-up (epoch, lists, body sums), marker kernel (records), the
    // tile-owned spread, then the force kernel (it needs only the marker
    // kernel's traction and body sums)
    e = launch_tile_begin(c, !clear, true);
    mark(1);
    if (e == cudaSuccess && before_marker) e = cudaStreamWaitEvent(c->stream, before_marker, 0);
    if (e == cudaSuccess)
      e = launch_mls_records(c, x, v, u, vv, w, p, accel, nullptr, c->d.fext, true, true, !clear);
    mark(2);
    if (e == cudaSuccess) e = launch_tile_spread(c, fx, fy, fz, !clear);
    mark(3);
    if (e == cudaSuccess)
      e = launch_force(c, x, v, c->d.fext, nullptr, x_out, v_out, nullptr, true, mirror);
    mark(4);
  } else {
    // the clear is a no-op for blocks that recorded no footprint (first step),
    // so it is launched unconditionally: a captured step then clears whatever
    // step ran before it.  It also zeroes the fixed-point body sums.
    e = clear ? launch_clear(c, fx, fy, fz) : zero_body_sums(c);
    mark(1);
    if (e == cudaSuccess && before_marker) e = cudaStreamWaitEvent(c->stream, before_marker, 0);
    if (e == cudaSuccess)
      e = launch_step_marker(c, x, v, u, vv, w, p, accel, fx, fy, fz, clear,
                             clear && !before_marker);
    mark(2);
    mark(3);
    if (e == cudaSuccess)
      e = launch_force(c, x, v, c->d.fext, nullptr, x_out, v_out, nullptr, true, mirror);
    mark(4);
  }
  if (e == cudaSuccess) {
    c->have_prev = clear;
    c->timed = c->timing;
  }
  return e;
}

// where a caller's array lives: device memory, page-locked host memory
// (reachable by the kernels at its device address) or other host memory
enum class Place { kDevice, kPinned, kOther };
Place place_of(const void* ptr, float** dev) {
  cudaPointerAttributes at{};
  *dev = nullptr;
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    cudaGetLastError();
    return Place::kOther;
  }
  *dev = static_cast<float*>(at.devicePointer);
  if (at.type == cudaMemoryTypeDevice) return Place::kDevice;
  if (at.type == cudaMemoryTypeHost && *dev) return Place::kPinned;
  return Place::kOther;
}

}  // namespace

extern "C" ibm_status ibm_step(ibm_ctx* c, const float* x, const float* v, const float* u,
                               const float* vv, const float* w, const float* p,
                               const float* accel, float* x_out, float* v_out, float* fx,
                               float* fy, float* fz, uint32_t flags) {
  if (!c || !x || !v || !u || !vv || !w || !x_out || !v_out || !fx || !fy || !fz)
    return set_err(c, IBM_ERR_INVALID_ARG, "null argument");
  if (x_out == x || v_out == v || x_out == v || v_out == x)
    return set_err(c, IBM_ERR_INVALID_ARG, "ibm_step: outputs must not alias the inputs");
  cudaSetDevice(c->device);
  return cuda_status(c, step_launches(c, x, v, u, vv, w, p, accel, x_out, v_out, fx, fy, fz,
                                      flags, nullptr),
                     "ibm_step");
}

extern "C" ibm_status ibm_step_host(ibm_ctx* c, const float* x, const float* v, const float* u,
                                    const float* vv, const float* w, const float* p,
                                    const float* accel, float* x_out, float* v_out, float* fx,
                                    float* fy, float* fz, uint32_t flags) {
  if (!c || !x || !v || !u || !vv || !w || !x_out || !v_out || !fx || !fy || !fz)
    return set_err(c, IBM_ERR_INVALID_ARG, "null argument");
  if (x_out == x || v_out == v || x_out == v || v_out == x)
    return set_err(c, IBM_ERR_INVALID_ARG, "ibm_step_host: outputs must not alias the inputs");
  cudaSetDevice(c->device);
  const size_t bytes = sizeof(float) * 3 * (size_t)c->V;
  if (!c->hcopy) {
    // all or nothing: the staging arrays, the copy stream and its events
    try {
      float* b[4];
      for (int k = 0; k < 4; ++k) b[k] = zeros<float>(c, 3 * (size_t)c->V);
      cudaStream_t st = nullptr;
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&e0, cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&e1, cudaEventDisableTiming);
      if (e != cudaSuccess) {
        if (st) cudaStreamDestroy(st);
        if (e0) cudaEventDestroy(e0);
        return cuda_status(c, e, "ibm_step_host");
      }
      int* cnt = zeros<int>(c, (3 * (size_t)c->V + kMirrorChunk - 1) / kMirrorChunk);
      for (int k = 0; k < 4; ++k) c->hs_buf[k] = b[k];
      c->hs_count = cnt;
      c->hcopy = st;
      c->ev_hfork = e0;
      c->ev_hcopy = e1;
    } catch (Failure& f) {
      return set_err(c, f.s, f.msg);
    }
  }
  // inputs: device arrays are used in place; host arrays are copied into the
  // staging arrays by the copy stream while the footprint clear runs (the
  // kernels gather positions by vertex id, which host memory serves poorly)
  float *xdv, *vdv, *xodv, *vodv;
  const Place px = place_of(x, &xdv), pv = place_of(v, &vdv);
  const Place pxo = place_of(x_out, &xodv), pvo = place_of(v_out, &vodv);
  const float* xd = px == Place::kDevice ? xdv : nullptr;
  const float* vd = pv == Place::kDevice ? vdv : nullptr;
  // outputs: device arrays written in place; page-locked host arrays (both)
  // mirrored chunk by chunk from the staging arrays by the force kernel,
  // whole 64-byte lines at a time, while it runs; otherwise staged and copied
  // back after the step
  Mirror mirror;
  float* xo = pxo == Place::kDevice ? xodv : nullptr;
  float* vo = pvo == Place::kDevice ? vodv : nullptr;
  if (pxo == Place::kPinned && pvo == Place::kPinned) {
    mirror.hx = xodv;
    mirror.hv = vodv;
    mirror.count = c->hs_count;
    mirror.vec = ((reinterpret_cast<uintptr_t>(xodv) | reinterpret_cast<uintptr_t>(vodv)) & 15u) == 0;
  }
  cudaError_t e = cudaSuccess;
  if (mirror.hx)
    e = cudaMemsetAsync(c->hs_count, 0,
                        sizeof(int) * ((3 * (size_t)c->V + kMirrorChunk - 1) / kMirrorChunk),
                        c->stream);
  cudaEvent_t join = nullptr;
  if (e == cudaSuccess && (!xd || !vd)) {
    e = cudaEventRecord(c->ev_hfork, c->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->hcopy, c->ev_hfork, 0);
    if (e == cudaSuccess && !xd)
      e = cudaMemcpyAsync(c->hs_buf[0], x, bytes, cudaMemcpyDefault, c->hcopy);
    if (e == cudaSuccess && !vd)
      e = cudaMemcpyAsync(c->hs_buf[1], v, bytes, cudaMemcpyDefault, c->hcopy);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_hcopy, c->hcopy);
    join = c->ev_hcopy;
  }
  if (e == cudaSuccess)
    e = step_launches(c, xd ? xd : c->hs_buf[0], vd ? vd : c->hs_buf[1], u, vv, w, p, accel,
                      xo ? xo : c->hs_buf[2], vo ? vo : c->hs_buf[3], fx, fy, fz, flags, join,
                      mirror.hx ? &mirror : nullptr);
  if (e == cudaSuccess && !xo && !mirror.hx)
    e = cudaMemcpyAsync(x_out, c->hs_buf[2], bytes, cudaMemcpyDefault, c->stream);
  if (e == cudaSuccess && !vo && !mirror.hx)
    e = cudaMemcpyAsync(v_out, c->hs_buf[3], bytes, cudaMemcpyDefault, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return cuda_status(c, e, "ibm_step_host");
}

// One loosely coupled time step (Sec. 5 steps 1-4): per RK3 substep the flow's
// predictor, the IBM forcing of the provisional velocity (marker kernel:
// interpolation at the centroids of x and spread of F = (V^b - U*)/dt, steps
// 3b-3d) and the pressure correction (3e); then the bodies advance with the
// probe traction and pressure of the new flow and the internal forces (4).
extern "C" ibm_status ibm_flow_step(ibm_flow* fl, ibm_ctx* c, const float* x, const float* xv,
                                    float* x_out, float* v_out, float* u, float* vv, float* w,
                                    float* p, float* fx, float* fy, float* fz) {
  auto bad = [&](const char* m) {
    set_global_error(m);
    return set_err(c, IBM_ERR_INVALID_ARG, m);
  };
  if (!fl || !u || !vv || !w || !p) return bad("ibm_flow_step: null argument");
  if (c) {
    if (!x || !xv || !x_out || !v_out || !fx || !fy || !fz) return bad("ibm_flow_step: null argument");
    if (x_out == x || v_out == xv || x_out == xv || v_out == x)
      return bad("ibm_flow_step: outputs must not alias the inputs");
    if (c->device != flow_device(fl)) return bad("ibm_flow_step: flow and context on different devices");
    if (!flow_matches(fl, c->gdesc, c->prm.dt, c->prm.mu))
      return bad("ibm_flow_step: the context's grid, dt and mu must equal the flow's grid, dt and nu");
  }
  cudaSetDevice(flow_device(fl));
  const cudaStream_t s = c ? c->stream : flow_stream(fl);
  const size_t cells = flow_cells(fl);
  cudaError_t e = cudaSuccess;
  if (c && !c->fc_tab) {
    // the forcing's cache and footprint record, allocated once
    try {
      const size_t nc = (size_t)std::max(c->n_chunks, 1);
      int2* rm = zeros<int2>(c, (size_t)kMaxRows * nc);
      int4* bx = zeros<int4>(c, 2 * nc);
      float4* fa = zeros<float4>(c, (size_t)2 * kMT * nc);
      c->fc_tab = zeros<int32_t>(c, (size_t)kCacheWords * nc);   // set last: marks all four
      c->fc_face = fa;
      c->fc_boxes = bx;
      c->fc_rowmap = rm;
    } catch (Failure& f) {
      set_global_error(f.msg);
      return set_err(c, f.s, f.msg);
    }
  }
  for (int l = 0; l < 3 && e == cudaSuccess; ++l) {
    e = flow_predict(fl, l, u, vv, w, p, s);
    if (c && e == cudaSuccess) {
      // substep 0 zeroes the fields; later substeps clear the previous
      // substep's footprint (inside launch_forcing)
      if (l == 0)
        for (float* f : {fx, fy, fz})
          if (e == cudaSuccess) e = cudaMemsetAsync(f, 0, cells * sizeof(float), s);
      if (e == cudaSuccess) e = launch_forcing(c, l, x, xv, u, vv, w, fx, fy, fz);
    }
    if (e == cudaSuccess)
      e = flow_project(fl, l, u, vv, w, p, c ? fx : nullptr, c ? fy : nullptr, c ? fz : nullptr,
                       c ? (float)c->prm.dt : 0.f, s);
  }
  if (c && e == cudaSuccess) {
    use_parity(c, c->qpar ^ 1);
    e = flow_mark_struct(fl, 0, s);
    if (e == cudaSuccess) e = zero_body_sums(c);
    if (e == cudaSuccess)
      e = launch_mls(c, x, nullptr, u, vv, w, p, nullptr, nullptr, nullptr, nullptr, c->d.fext,
                     nullptr, nullptr, nullptr, true, false, true, false, false);
    if (e == cudaSuccess) e = flow_mark_struct(fl, 1, s);
    if (e == cudaSuccess) e = launch_force(c, x, xv, c->d.fext, nullptr, x_out, v_out, nullptr, true);
    if (e == cudaSuccess) e = flow_mark_struct(fl, 2, s);
  }
  if (e != cudaSuccess) {
    const std::string m = std::string("ibm_flow_step: ") + cudaGetErrorString(e);
    set_global_error(m);
    return set_err(c, IBM_ERR_CUDA, m);
  }
  return IBM_OK;
}

namespace {

// acceleration a = (F_int + F_ext^v)/m at positions x: body sums, probe
// traction (the marker kernel's measure and probe parts) and the force
// kernel in its acceleration mode
cudaError_t eval_accel(ibm_ctx* c, const float* x, const float* u, const float* vv,
                       const float* w, const float* p, const float* accel, float* a) {
  cudaError_t e = zero_body_sums(c);
  if (e == cudaSuccess)
    e = launch_mls(c, x, nullptr, u, vv, w, p, accel, nullptr, nullptr, nullptr, c->d.fext, nullptr,
                   nullptr, nullptr, true, false, true, false, false);
  if (e == cudaSuccess) e = launch_accel(c, x, c->d.fext, a);
  return e;
}

void pc_allocate(ibm_ctx* c) {
  auto& P = c->pc;
  if (P.pcx) return;
  const size_t n = 3 * (size_t)c->V;
  for (int k = 0; k < 3; ++k) {
    P.yx[k] = zeros<float>(c, n);
    P.yv[k] = zeros<float>(c, n);
    P.a[k] = zeros<float>(c, n);
  }
  P.pcx = zeros<float>(c, n);
  P.pcv = zeros<float>(c, n);
  P.px = zeros<float>(c, n);
  P.pv = zeros<float>(c, n);
  P.mx = zeros<float>(c, n);
  P.mv = zeros<float>(c, n);
  P.am = zeros<float>(c, n);
  P.sx = zeros<float>(c, n);
  P.v2 = zeros<float>(c, n);
  P.v3 = zeros<float>(c, n);
  P.v4 = zeros<float>(c, n);
  P.a2 = zeros<float>(c, n);
  P.a3 = zeros<float>(c, n);
  P.a4 = zeros<float>(c, n);
}

LinComb lc(std::initializer_list<std::pair<float, const float*>> terms) {
  LinComb L{};
  for (const auto& t : terms) {
    L.c[L.k] = t.first;
    L.in[L.k] = t.second;
    ++L.k;
  }
  return L;
}

}  // namespace

extern "C" ibm_status ibm_pc_reset(ibm_ctx* c) {
  if (!c) return IBM_ERR_INVALID_ARG;
  c->pc.steps = 0;
  c->pc.have_pc = false;
  return IBM_OK;
}

namespace {

// Checkpoint of the context's own mutable state (ibm_get_state/ibm_set_state):
// a fixed header, then the strong-coupling history (when steps > 0: ten
// [3][V] float arrays), then the footprint record of the spread variant in
// use (1: every marker patch's two box words and its rows, compacted to the
// rows the box declares; 2: every tile's clear-mode epoch and nonzero-segment
// mask).  Host byte order.
struct StateHeader {
  char magic[8];          // "IBMSTATE"
  uint32_t version;       // 1
  int32_t spread_variant;
  int64_t V, F, n_chunks, n_tiles;
  int32_t grid_n[3];      // grid nodes per direction
  uint32_t dt_bits;       // the step size the history belongs to
  int32_t pc_steps;       // ibm_step_pc calls since ibm_pc_reset
  int32_t pc_have;        // the last step's predictor-corrector difference is held
  int32_t tile_epoch;     // clear-mode epoch of the tile-owned spread
  int32_t reserved;       // 0
  int64_t n_rows;         // row records of the variant-1 footprint
};
static_assert(sizeof(StateHeader) == 88, "state header layout");
constexpr char kStateMagic[8] = {'I', 'B', 'M', 'S', 'T', 'A', 'T', 'E'};
constexpr int kStateArrays = 10;

// the history arrays in their logical order: y_{n-1..n-3} (x, then v), a_n,
// a_{n-1} as the next step sees them, and p - c of the last step
void state_arrays(ibm_ctx* c, float* (&out)[kStateArrays]) {
  auto& P = c->pc;
  float* a[kStateArrays] = {P.yx[0], P.yx[1], P.yx[2], P.yv[0], P.yv[1],
                            P.yv[2], P.a[1],  P.a[2],  P.pcx,   P.pcv};
  for (int k = 0; k < kStateArrays; ++k) out[k] = a[k];
}

// rows a variant-1 box declares (what the clear kernel reads of its rows)
int64_t box_rows(const int4& lo, const int4& sz) {
  if (sz.x <= 0 || sz.y <= 0 || sz.z <= 0 || lo.w == 1) return 0;
  return std::max(sz.w, 0);
}

// a footprint record from a checkpoint may only name nodes of this grid
bool box_valid(const ibm_ctx* c, const int4& lo, const int4& sz) {
  if (lo.w < 0 || lo.w > 2) return false;
  // corners well inside int range (the clear wraps lo + offset into the grid)
  const int lim = 1 << 28;
  if (std::abs(lo.x) > lim || std::abs(lo.y) > lim || std::abs(lo.z) > lim) return false;
  if (sz.x > c->grid.n[0] || sz.y > c->grid.n[1] || sz.z > c->grid.n[2]) return false;
  return sz.w >= 0 && sz.w <= kMaxRows;
}

bool row_valid(const ibm_ctx* c, const int2& e) {
  const int L = e.y >> 16, x0 = e.y & 0xFFFF;
  if (L <= 0) return true;   // skipped by the clear
  const int64_t nx = c->grid.n[0];
  const int64_t total = nx * c->grid.n[1] * c->grid.n[2];
  return L <= nx && x0 < nx && e.x >= 0 && e.x % nx == 0 && (int64_t)e.x < total;
}

}  // namespace

extern "C" ibm_status ibm_get_state(ibm_ctx* c, void* buf, int64_t capacity, int64_t* size) {
  if (!c || !size) return set_err(c, IBM_ERR_INVALID_ARG, "null argument");
  const ibm_status st = ibm_check_device_error(c);
  if (st != IBM_OK) return st;
  cudaSetDevice(c->device);
  StateHeader h{};
  std::memcpy(h.magic, kStateMagic, sizeof(h.magic));
  h.version = 1;
  h.spread_variant = c->spread_variant;
  h.V = c->V;
  h.F = c->F;
  h.n_chunks = c->n_chunks;
  h.n_tiles = c->spread_variant == 2 ? c->td.n_tiles : 0;
  for (int k = 0; k < 3; ++k) h.grid_n[k] = c->grid.n[k];
  std::memcpy(&h.dt_bits, &c->sc.dt, sizeof(h.dt_bits));
  h.pc_steps = c->pc.pcx ? c->pc.steps : 0;
  h.pc_have = h.pc_steps > 0 && c->pc.have_pc ? 1 : 0;
  cudaError_t e = cudaSuccess;
  std::vector<int4> boxes;
  std::vector<int2> rows;
  if (c->spread_variant == 2) {
    e = cudaMemcpy(&h.tile_epoch, c->td.state + TS_EPOCH, sizeof(int32_t), cudaMemcpyDeviceToHost);
  } else if (c->n_chunks > 0) {
    boxes.resize(2 * (size_t)c->n_chunks);
    rows.resize((size_t)kMaxRows * c->n_chunks);
    e = cudaMemcpy(boxes.data(), c->d.boxes, sizeof(int4) * boxes.size(), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
      e = cudaMemcpy(rows.data(), c->d.rowmap, sizeof(int2) * rows.size(), cudaMemcpyDeviceToHost);
    // compact: each patch's declared rows, in patch order
    size_t n = 0;
    for (int64_t q = 0; q < c->n_chunks && e == cudaSuccess; ++q) {
      const int64_t r = box_rows(boxes[2 * q], boxes[2 * q + 1]);
      std::memmove(rows.data() + n, rows.data() + (size_t)q * kMaxRows, sizeof(int2) * r);
      n += (size_t)r;
    }
    rows.resize(n);
    h.n_rows = (int64_t)n;
  }
  if (e != cudaSuccess) return cuda_status(c, e, "ibm_get_state");
  const int64_t hist = h.pc_steps > 0 ? (int64_t)kStateArrays * 3 * c->V * 4 : 0;
  const int64_t total = (int64_t)sizeof(h) + hist +
                        (c->spread_variant == 2
                             ? 13 * 4 * h.n_tiles
                             : (int64_t)sizeof(int4) * (int64_t)boxes.size() + 8 * h.n_rows);
  *size = total;
  if (!buf) return IBM_OK;
  if (capacity < total)
    return set_err(c, IBM_ERR_INVALID_ARG,
                   "ibm_get_state: the buffer holds " + std::to_string(capacity) +
                       " bytes, the state needs " + std::to_string(total));
  char* o = static_cast<char*>(buf);
  std::memcpy(o, &h, sizeof(h));
  o += sizeof(h);
  if (hist) {
    float* a[kStateArrays];
    state_arrays(c, a);
    const size_t bytes = sizeof(float) * 3 * (size_t)c->V;
    for (int k = 0; k < kStateArrays && e == cudaSuccess; ++k, o += bytes)
      e = cudaMemcpy(o, a[k], bytes, cudaMemcpyDeviceToHost);
  }
  if (e == cudaSuccess && c->spread_variant == 2 && h.n_tiles > 0) {
    e = cudaMemcpy(o, c->td.epoch, 4 * (size_t)h.n_tiles, cudaMemcpyDeviceToHost);
    o += 4 * (size_t)h.n_tiles;
    if (e == cudaSuccess)
      e = cudaMemcpy(o, c->td.mask, 48 * (size_t)h.n_tiles, cudaMemcpyDeviceToHost);
  } else if (c->spread_variant != 2) {
    std::memcpy(o, boxes.data(), sizeof(int4) * boxes.size());
    o += sizeof(int4) * boxes.size();
    std::memcpy(o, rows.data(), sizeof(int2) * rows.size());
  }
  return cuda_status(c, e, "ibm_get_state");
}

extern "C" ibm_status ibm_set_state(ibm_ctx* c, const void* buf, int64_t size) {
  if (!c || !buf) return set_err(c, IBM_ERR_INVALID_ARG, "null argument");
  auto bad = [c](const std::string& m) {
    return set_err(c, IBM_ERR_INVALID_ARG, "ibm_set_state: " + m);
  };
  if (size < (int64_t)sizeof(StateHeader)) return bad("truncated state");
  StateHeader h;
  std::memcpy(&h, buf, sizeof(h));
  if (std::memcmp(h.magic, kStateMagic, sizeof(h.magic)) != 0 || h.version != 1)
    return bad("not a state of this library");
  uint32_t dt_bits;
  std::memcpy(&dt_bits, &c->sc.dt, sizeof(dt_bits));
  const int64_t n_tiles = c->spread_variant == 2 ? c->td.n_tiles : 0;
  if (h.spread_variant != c->spread_variant || h.V != c->V || h.F != c->F ||
      h.n_chunks != c->n_chunks || h.n_tiles != n_tiles || h.dt_bits != dt_bits ||
      h.grid_n[0] != c->grid.n[0] || h.grid_n[1] != c->grid.n[1] || h.grid_n[2] != c->grid.n[2])
    return bad("the state belongs to a context of other bodies, grid, parameters or spread "
               "variant");
  if (h.pc_steps < 0 || (h.pc_have != 0 && h.pc_have != 1) || h.reserved != 0 || h.n_rows < 0 ||
      h.n_rows > (int64_t)kMaxRows * c->n_chunks || (c->spread_variant == 2 && h.n_rows != 0))
    return bad("corrupt header");
  const int64_t hist = h.pc_steps > 0 ? (int64_t)kStateArrays * 3 * c->V * 4 : 0;
  const int64_t total = (int64_t)sizeof(h) + hist +
                        (c->spread_variant == 2 ? 13 * 4 * n_tiles
                                                : 32 * (int64_t)c->n_chunks + 8 * h.n_rows);
  if (size != total) return bad("size does not match the header");
  const char* in = static_cast<const char*>(buf) + sizeof(h);
  const char* rec = in + hist;
  // check the footprint record before anything reaches the device: the next
  // clear-mode step writes zeros where it points
  std::vector<int2> rowmap;
  if (c->spread_variant != 2 && c->n_chunks > 0) {
    std::vector<int4> boxes(2 * (size_t)c->n_chunks);
    std::memcpy(boxes.data(), rec, sizeof(int4) * boxes.size());
    const char* rp = rec + sizeof(int4) * boxes.size();
    rowmap.assign((size_t)kMaxRows * c->n_chunks, make_int2(0, 0));
    int64_t n = 0;
    for (int64_t q = 0; q < c->n_chunks; ++q) {
      if (!box_valid(c, boxes[2 * q], boxes[2 * q + 1])) return bad("corrupt footprint box");
      const int64_t r = box_rows(boxes[2 * q], boxes[2 * q + 1]);
      if (n + r > h.n_rows) return bad("footprint rows do not match the header");
      std::memcpy(rowmap.data() + (size_t)q * kMaxRows, rp + 8 * n, 8 * (size_t)r);
      for (int64_t k = 0; k < r; ++k)
        if (!row_valid(c, rowmap[(size_t)q * kMaxRows + k])) return bad("corrupt footprint row");
      n += r;
    }
    if (n != h.n_rows) return bad("footprint rows do not match the header");
  }
  cudaSetDevice(c->device);
  if (h.pc_steps > 0) {
    try {
      pc_allocate(c);
    } catch (Failure& f) {
      return set_err(c, f.s, f.msg);
    }
  }
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (hist && e == cudaSuccess) {
    float* a[kStateArrays];
    state_arrays(c, a);
    const size_t bytes = sizeof(float) * 3 * (size_t)c->V;
    for (int k = 0; k < kStateArrays && e == cudaSuccess; ++k)
      e = cudaMemcpy(a[k], in + k * bytes, bytes, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess && c->spread_variant == 2 && n_tiles > 0) {
    e = cudaMemcpy(c->td.state + TS_EPOCH, &h.tile_epoch, sizeof(int32_t),
                   cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(c->td.epoch, rec, 4 * (size_t)n_tiles, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(c->td.mask, rec + 4 * (size_t)n_tiles, 48 * (size_t)n_tiles,
                     cudaMemcpyHostToDevice);
  } else if (e == cudaSuccess && c->spread_variant != 2 && c->n_chunks > 0) {
    e = cudaMemcpy(c->d.boxes, rec, 32 * (size_t)c->n_chunks, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(c->d.rowmap, rowmap.data(), sizeof(int2) * rowmap.size(),
                     cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) return cuda_status(c, e, "ibm_set_state");
  c->pc.steps = h.pc_steps;
  c->pc.have_pc = h.pc_have != 0;
  return IBM_OK;
}

extern "C" ibm_status ibm_step_pc(ibm_ctx* c, const float* x, const float* v, const float* u,
                                  const float* vv, const float* w, const float* p,
                                  const float* accel, float* x_out, float* v_out, float* fx,
                                  float* fy, float* fz, uint32_t flags) {
  if (!c || !x || !v || !u || !vv || !w || !x_out || !v_out || !fx || !fy || !fz)
    return set_err(c, IBM_ERR_INVALID_ARG, "null argument");
  if (x_out == x || v_out == v || x_out == v || v_out == x)
    return set_err(c, IBM_ERR_INVALID_ARG, "ibm_step_pc: outputs must not alias the inputs");
  cudaSetDevice(c->device);
  try {
    pc_allocate(c);
  } catch (Failure& f) {
    return set_err(c, f.s, f.msg);
  }
  auto& P = c->pc;
  const float h = c->sc.dt;
  const bool clear = (flags & IBM_STEP_CLEAR_PREV) != 0;
  use_parity(c, c->qpar ^ 1);
  // at y_n: footprint clear, interpolation, spreading, probe traction, body
  // sums (as ibm_step), then a_n
  cudaError_t e = cudaSuccess;
  if (c->spread_variant == 2) {
    e = launch_tile_begin(c, !clear, true);
    if (e == cudaSuccess)
      e = launch_mls_records(c, x, v, u, vv, w, p, accel, nullptr, c->d.fext, true, true, !clear);
    if (e == cudaSuccess) e = launch_tile_spread(c, fx, fy, fz, !clear);
  } else {
    e = clear ? launch_clear(c, fx, fy, fz) : zero_body_sums(c);
    if (e == cudaSuccess)
      e = launch_step_marker(c, x, v, u, vv, w, p, accel, fx, fy, fz, clear, clear);
  }
  float* an = P.a[0];
  if (e == cudaSuccess) e = launch_accel(c, x, c->d.fext, an);
  if (P.steps < 3) {
    // classical Runge-Kutta start-up: k_i = (v_i, a_i)
    if (e == cudaSuccess) e = launch_lincomb(c, P.sx, lc({{1.f, x}, {0.5f * h, v}}));
    if (e == cudaSuccess) e = launch_lincomb(c, P.v2, lc({{1.f, v}, {0.5f * h, an}}));
    if (e == cudaSuccess) e = eval_accel(c, P.sx, u, vv, w, p, accel, P.a2);
    if (e == cudaSuccess) e = launch_lincomb(c, P.sx, lc({{1.f, x}, {0.5f * h, P.v2}}));
    if (e == cudaSuccess) e = launch_lincomb(c, P.v3, lc({{1.f, v}, {0.5f * h, P.a2}}));
    if (e == cudaSuccess) e = eval_accel(c, P.sx, u, vv, w, p, accel, P.a3);
    if (e == cudaSuccess) e = launch_lincomb(c, P.sx, lc({{1.f, x}, {h, P.v3}}));
    if (e == cudaSuccess) e = launch_lincomb(c, P.v4, lc({{1.f, v}, {h, P.a3}}));
    if (e == cudaSuccess) e = eval_accel(c, P.sx, u, vv, w, p, accel, P.a4);
    const float s = h / 6.f;
    if (e == cudaSuccess)
      e = launch_lincomb(c, x_out, lc({{1.f, x}, {s, v}, {2.f * s, P.v2}, {2.f * s, P.v3},
                                       {s, P.v4}}));
    if (e == cudaSuccess)
      e = launch_lincomb(c, v_out, lc({{1.f, v}, {s, an}, {2.f * s, P.a2}, {2.f * s, P.a3},
                                       {s, P.a4}}));
    P.have_pc = false;
  } else {
    HamPredict Pr{};
    Pr.x3 = P.yx[2];
    Pr.v3 = P.yv[2];
    Pr.vn = v;
    Pr.vn1 = P.yv[0];
    Pr.vn2 = P.yv[1];
    Pr.an = an;
    Pr.an1 = P.a[1];
    Pr.an2 = P.a[2];
    Pr.pcx = P.pcx;
    Pr.pcv = P.pcv;
    Pr.px = P.px;
    Pr.pv = P.pv;
    Pr.mx = P.mx;
    Pr.mv = P.mv;
    Pr.h = h;
    Pr.first = P.have_pc ? 0 : 1;
    if (e == cudaSuccess) e = launch_ham_predict(c, Pr);
    if (e == cudaSuccess) e = eval_accel(c, P.mx, u, vv, w, p, accel, P.am);
    HamCorrect Co{};
    Co.xn = x;
    Co.vn = v;
    Co.x2 = P.yx[1];
    Co.v2 = P.yv[1];
    Co.vn1 = P.yv[0];
    Co.an = an;
    Co.an1 = P.a[1];
    Co.mv = P.mv;
    Co.am = P.am;
    Co.px = P.px;
    Co.pv = P.pv;
    Co.clamp = c->d.clamp;
    Co.xo = x_out;
    Co.vo = v_out;
    Co.pcx = P.pcx;
    Co.pcv = P.pcv;
    Co.h = h;
    if (e == cudaSuccess) e = launch_ham_correct(c, Co);
    P.have_pc = true;
  }
  // history: y_n joins the ring (its oldest buffer is reused), a_n likewise
  if (e == cudaSuccess) {
    float* ox = P.yx[2];
    float* ov = P.yv[2];
    P.yx[2] = P.yx[1];
    P.yv[2] = P.yv[1];
    P.yx[1] = P.yx[0];
    P.yv[1] = P.yv[0];
    P.yx[0] = ox;
    P.yv[0] = ov;
    const size_t bytes = sizeof(float) * 3 * (size_t)c->V;
    e = cudaMemcpyAsync(ox, x, bytes, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ov, v, bytes, cudaMemcpyDeviceToDevice, c->stream);
    float* oa = P.a[2];
    P.a[2] = P.a[1];
    P.a[1] = P.a[0];
    P.a[0] = oa;
    ++P.steps;
    c->have_prev = clear;
  }
  return cuda_status(c, e, "ibm_step_pc");
}

struct ibm_graph {
  ibm_ctx* ctx = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

extern "C" ibm_status ibm_graph_create(ibm_ctx* c, float* xa, float* va, float* xb, float* vb,
                                       const float* u, const float* vv, const float* w,
                                       const float* p, const float* accel, float* fx, float* fy,
                                       float* fz, int32_t n_steps, ibm_graph** out) {
  if (out) *out = nullptr;
  if (!c || !xa || !va || !xb || !vb || !u || !vv || !w || !fx || !fy || !fz || !out)
    return set_err(c, IBM_ERR_INVALID_ARG, "null argument");
  if (n_steps < 2 || (n_steps & 1))
    return set_err(c, IBM_ERR_INVALID_ARG, "ibm_graph_create: n_steps must be even and >= 2");
  cudaSetDevice(c->device);
  cudaStream_t cap = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_status(c, e, "cudaStreamCreate");
  // order the capture after work already queued on the context's stream
  cudaEvent_t ready = nullptr;
  e = cudaEventCreateWithFlags(&ready, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(ready, c->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cap, ready, 0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cap);
  if (ready) cudaEventDestroy(ready);
  if (e != cudaSuccess) {
    cudaStreamDestroy(cap);
    return cuda_status(c, e, "ibm_graph_create");
  }
  const cudaStream_t saved = c->stream;
  const bool timing = c->timing;
  c->stream = cap;
  c->timing = false;
  ibm_graph* g = new ibm_graph();
  g->ctx = c;
  ibm_status st = IBM_OK;
  // A side stream carries each step's clear of the previous footprint: inside
  // the graph the force fields of intermediate steps are never observed, so
  // step k+1's clear runs concurrently with step k's force kernel (it needs
  // only step k's recorded footprint); step k+1's marker kernel waits for it.
  cudaStream_t side = nullptr;
  cudaEvent_t ev_marker = nullptr, ev_clear = nullptr;
  e = cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_marker, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_clear, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess && c->spread_variant == 2) {
    // per step: set-up, marker kernel; then the force kernel on the capture
    // stream while the tile-owned spread runs on the side stream (the two are
    // independent: the spread reads the records, the force kernel the traction
    // and body sums); the next step waits for both
    for (int k = 0; k < n_steps && e == cudaSuccess; ++k) {
      const bool even = (k & 1) == 0;
      const float* x = even ? xa : xb;
      const float* v = even ? va : vb;
      use_parity(c, c->qpar ^ 1);
      e = launch_tile_begin(c, false, true);
      if (e == cudaSuccess)
        e = launch_mls_records(c, x, v, u, vv, w, p, accel, nullptr, c->d.fext, true, true, false);
      if (e == cudaSuccess) e = cudaEventRecord(ev_marker, cap);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(side, ev_marker, 0);
      if (e == cudaSuccess) {
        c->stream = side;
        e = launch_tile_spread(c, fx, fy, fz, false);
        c->stream = cap;
      }
      if (e == cudaSuccess) e = cudaEventRecord(ev_clear, side);
      if (e == cudaSuccess)
        e = launch_force(c, x, v, c->d.fext, nullptr, even ? xb : xa, even ? vb : va, nullptr,
                         true);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(cap, ev_clear, 0);
    }
    if (e != cudaSuccess) st = cuda_status(c, e, "ibm_graph_create");
    cudaGraph_t graph = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
    if (e2 == cudaSuccess && st == IBM_OK) {
      g->graph = graph;
      e = cudaGraphInstantiate(&g->exec, graph, 0);
    } else {
      if (graph) cudaGraphDestroy(graph);
      e = e2;
    }
  } else if (e == cudaSuccess) {
    for (int k = 0; k < n_steps && e == cudaSuccess; ++k) {
      const bool even = (k & 1) == 0;
      const float* x = even ? xa : xb;
      const float* v = even ? va : vb;
      use_parity(c, c->qpar ^ 1);
      // step 0's marker kernel overlaps the clear just before it; the later
      // steps' follow the previous force kernel, with their clear on the side
      if (k == 0) e = launch_clear(c, fx, fy, fz);
      if (e == cudaSuccess)
        e = launch_step_marker(c, x, v, u, vv, w, p, accel, fx, fy, fz, true, k == 0);
      const bool next = k + 1 < n_steps;
      if (next && e == cudaSuccess) {
        e = cudaEventRecord(ev_marker, cap);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(side, ev_marker, 0);
        // the next step's clear, with the next step's body-sum buffer
        const int p = c->qpar;
        c->stream = side;
        use_parity(c, p ^ 1);
        if (e == cudaSuccess) e = launch_clear(c, fx, fy, fz);
        use_parity(c, p);
        c->stream = cap;
        if (e == cudaSuccess) e = cudaEventRecord(ev_clear, side);
      }
      if (e == cudaSuccess)
        e = launch_force(c, x, v, c->d.fext, nullptr, even ? xb : xa, even ? vb : va, nullptr,
                         true);
      if (next && e == cudaSuccess) e = cudaStreamWaitEvent(cap, ev_clear, 0);
    }
    if (e != cudaSuccess) st = cuda_status(c, e, "ibm_graph_create");
    cudaGraph_t graph = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
    if (e2 == cudaSuccess && st == IBM_OK) {
      g->graph = graph;
      e = cudaGraphInstantiate(&g->exec, graph, 0);
    } else {
      if (graph) cudaGraphDestroy(graph);
      e = e2;
    }
  }
  c->stream = saved;
  c->timing = timing;
  if (st == IBM_OK && e == cudaSuccess) c->have_prev = true;
  cudaStreamDestroy(cap);
  if (side) cudaStreamDestroy(side);
  if (ev_marker) cudaEventDestroy(ev_marker);
  if (ev_clear) cudaEventDestroy(ev_clear);
  if (st != IBM_OK || e != cudaSuccess) {
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    return st != IBM_OK ? st : cuda_status(c, e, "ibm_graph_create");
  }
  *out = g;
  return IBM_OK;
}

extern "C" ibm_status ibm_graph_launch(ibm_graph* g) {
  if (!g || !g->exec) return IBM_ERR_INVALID_ARG;
  cudaSetDevice(g->ctx->device);
  return cuda_status(g->ctx, cudaGraphLaunch(g->exec, g->ctx->stream), "ibm_graph_launch");
}

extern "C" void ibm_graph_destroy(ibm_graph* g) {
  if (!g) return;
  cudaSetDevice(g->ctx->device);
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  delete g;
}

extern "C" ibm_status ibm_set_phase_timing(ibm_ctx* c, int32_t on) {
  if (!c) return IBM_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  if (on && !c->ev[0]) {
    for (auto& ev : c->ev) {
      cudaError_t e = cudaEventCreate(&ev);
      if (e != cudaSuccess) return cuda_status(c, e, "cudaEventCreate");
    }
  }
  c->timing = on != 0;
  c->timed = false;
  return IBM_OK;
}

extern "C" ibm_status ibm_get_counters(ibm_ctx* c, int64_t* out) {
  if (!c || !out) return set_err(c, IBM_ERR_INVALID_ARG, "null argument");
  cudaSetDevice(c->device);
  int32_t s[4] = {0, 0, 0, 0};
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess) e = cudaMemcpy(s, c->d.stats, sizeof(s), cudaMemcpyDeviceToHost);
  for (int k = 0; k < 4; ++k) out[k] = s[k];
  return cuda_status(c, e, "ibm_get_counters");
}

extern "C" ibm_status ibm_get_phase_times(ibm_ctx* c, float* ms) {
  if (!c || !ms) return set_err(c, IBM_ERR_INVALID_ARG, "null argument");
  if (!c->timed) return set_err(c, IBM_ERR_INVALID_ARG, "no timed ibm_step recorded");
  cudaSetDevice(c->device);
  cudaError_t e = cudaEventSynchronize(c->ev[4]);
  for (int k = 0; k < 4 && e == cudaSuccess; ++k) e = cudaEventElapsedTime(ms + k, c->ev[k], c->ev[k + 1]);
  return cuda_status(c, e, "ibm_get_phase_times");
}

extern "C" ibm_status ibm_backward(ibm_ctx* c, const float* x, const float* v, const float* u,
                                   const float* vv, const float* w, const float* p,
                                   const float* accel, const float* gx_next, const float* gv_next,
                                   const float* gfx, const float* gfy, const float* gfz, float* gx,
                                   float* gv, double* gparams) {
  if (!c || !x || !u || !vv || !w || !gx_next || !gv_next || !gx || !gv || !gparams)
    return set_err(c, IBM_ERR_INVALID_ARG, "null argument");
  if (gx == gx_next || gv == gv_next || gx == gv_next || gv == gx_next)
    return set_err(c, IBM_ERR_INVALID_ARG, "ibm_backward: outputs must not alias the cotangents");
  const int ngf = (gfx ? 1 : 0) + (gfy ? 1 : 0) + (gfz ? 1 : 0);
  if (ngf != 0 && ngf != 3)
    return set_err(c, IBM_ERR_INVALID_ARG, "ibm_backward: give all three field cotangents or none");
  if (ngf == 3 && !v)
    return set_err(c, IBM_ERR_INVALID_ARG,
                   "ibm_backward: the spread's cotangent needs the vertex velocities v");
  cudaSetDevice(c->device);
  return cuda_status(c, launch_backward(c, x, v, u, vv, w, p, accel, gx_next, gv_next, gfx, gfy,
                                       gfz, gx, gv, gparams),
                     "ibm_backward");
}

extern "C" ibm_status ibm_taylor_deformation(ibm_ctx* c, const float* x, double* D) {
  if (!c || !x || !D) return set_err(c, IBM_ERR_INVALID_ARG, "null argument");
  cudaSetDevice(c->device);
  return cuda_status(c, launch_taylor(c, x, D), "ibm_taylor_deformation");
}

extern "C" ibm_status ibm_taylor_backward(ibm_ctx* c, const float* x, const double* gD, float* gx,
                                          double* D) {
  if (!c || !x || !gD || !gx || !D) return set_err(c, IBM_ERR_INVALID_ARG, "null argument");
  cudaSetDevice(c->device);
  cudaError_t e = launch_taylor(c, x, D);
  if (e == cudaSuccess) e = launch_taylor_backward(c, x, gD, gx);
  return cuda_status(c, e, "ibm_taylor_backward");
}

extern "C" ibm_status ibm_check_device_error(ibm_ctx* c) {
  if (!c) return IBM_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  int32_t w = 0;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess) e = cudaMemcpy(&w, c->d.err, sizeof(w), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_status(c, e, "ibm_check_device_error");
  if (w) {
    cudaMemset(c->d.err, 0, sizeof(w));
    return set_err(c, IBM_ERR_DEVICE,
                   std::string("device error word ") + std::to_string(w) +
                       ((w & ERR_NONFINITE) ? " (non-finite or out-of-range marker position)" : "") +
                       ((w & ERR_TILE_DENSE) ? " (more than 65535 markers reach one spread tile)"
                                             : "") +
                       ((w & ERR_TIMEOUT) ? " (a wait for a bulk copy into shared memory ran out)"
                                          : ""));
  }
  return IBM_OK;
}
