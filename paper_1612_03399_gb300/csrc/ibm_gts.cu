// GTS (GNU Triangulated Surface) import: the text format in which the
// paper's Lagrangian meshes are exported (Sec. 5): a header "nv ne nf", nv
// vertex lines "x y z", ne edge lines of two 1-based vertex indices and nf
// face lines of three 1-based edge indices.  A face's vertex order follows
// its edges: the vertex of e1 not on e2, the vertex e1 and e2 share, then the
// vertex of e2 not on e1.  Host code only; no device is needed.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "ibm_internal.cuh"

namespace {

// next line that is not empty and not a comment ('#'), or false at the end
bool next_line(FILE* f, std::string& line) {
  char buf[4096];
  while (std::fgets(buf, sizeof(buf), f)) {
    size_t n = std::strlen(buf);
    line.assign(buf, n);
    // a line longer than the buffer: keep reading it
    while (n > 0 && buf[n - 1] != '\n' && std::fgets(buf, sizeof(buf), f)) {
      n = std::strlen(buf);
      line.append(buf, n);
    }
    size_t i = 0;
    while (i < line.size() && (line[i] == ' ' || line[i] == '\t' || line[i] == '\r' ||
                               line[i] == '\n'))
      ++i;
    if (i == line.size() || line[i] == '#') continue;
    return true;
  }
  return false;
}

struct Gts {
  std::vector<double> xyz;
  std::vector<int32_t> tri;
};

ibm_status fail(const std::string& m, ibm_status s) {
  ibm::set_global_error(m);
  return s;
}

ibm_status parse(const char* path, Gts& out) {
  FILE* f = std::fopen(path, "r");
  if (!f) return fail(std::string("ibm_gts_read: cannot open ") + path, IBM_ERR_INVALID_ARG);
  std::string line;
  long long nv = -1, ne = -1, nf = -1;
  ibm_status st = IBM_OK;
  std::string msg;
  auto bad = [&](const std::string& m, ibm_status s) {
    msg = m;
    st = s;
  };
  if (!next_line(f, line) || std::sscanf(line.c_str(), "%lld %lld %lld", &nv, &ne, &nf) != 3 ||
      nv < 3 || ne < 3 || nf < 1 || nv > (1ll << 30) || ne > (1ll << 30) || nf > (1ll << 30)) {
    bad("ibm_gts_read: the first line must hold the counts nv ne nf", IBM_ERR_INVALID_ARG);
  }
  std::vector<int64_t> edge;
  if (st == IBM_OK) {
    out.xyz.resize(3 * (size_t)nv);
    for (long long i = 0; i < nv && st == IBM_OK; ++i) {
      double* p = &out.xyz[3 * (size_t)i];
      if (!next_line(f, line) || std::sscanf(line.c_str(), "%lf %lf %lf", p, p + 1, p + 2) != 3)
        bad("ibm_gts_read: vertex line " + std::to_string(i + 1) + " is not 'x y z'",
            IBM_ERR_INVALID_ARG);
    }
  }
  if (st == IBM_OK) {
    edge.resize(2 * (size_t)ne);
    for (long long i = 0; i < ne && st == IBM_OK; ++i) {
      long long a = 0, b = 0;
      if (!next_line(f, line) || std::sscanf(line.c_str(), "%lld %lld", &a, &b) != 2) {
        bad("ibm_gts_read: edge line " + std::to_string(i + 1) + " is not two indices",
            IBM_ERR_INVALID_ARG);
      } else if (a < 1 || b < 1 || a > nv || b > nv || a == b) {
        bad("ibm_gts_read: edge " + std::to_string(i + 1) + " has a bad vertex index",
            IBM_ERR_MESH);
      } else {
        edge[2 * i] = a - 1;
        edge[2 * i + 1] = b - 1;
      }
    }
  }
  if (st == IBM_OK) {
    out.tri.resize(3 * (size_t)nf);
    for (long long i = 0; i < nf && st == IBM_OK; ++i) {
      long long e[3] = {0, 0, 0};
      if (!next_line(f, line) || std::sscanf(line.c_str(), "%lld %lld %lld", e, e + 1, e + 2) != 3) {
        bad("ibm_gts_read: face line " + std::to_string(i + 1) + " is not three indices",
            IBM_ERR_INVALID_ARG);
        break;
      }
      bool ok = true;
      for (int k = 0; k < 3; ++k) ok = ok && e[k] >= 1 && e[k] <= ne;
      if (!ok) {
        bad("ibm_gts_read: face " + std::to_string(i + 1) + " has a bad edge index", IBM_ERR_MESH);
        break;
      }
      const int64_t a0 = edge[2 * (e[0] - 1)], a1 = edge[2 * (e[0] - 1) + 1];
      const int64_t b0 = edge[2 * (e[1] - 1)], b1 = edge[2 * (e[1] - 1) + 1];
      const int64_t c0 = edge[2 * (e[2] - 1)], c1 = edge[2 * (e[2] - 1) + 1];
      // v2 = the vertex e1 and e2 share
      int64_t v1, v2, v3;
      if (a1 == b0 || a1 == b1) {
        v1 = a0;
        v2 = a1;
      } else if (a0 == b0 || a0 == b1) {
        v1 = a1;
        v2 = a0;
      } else {
        bad("ibm_gts_read: the first two edges of face " + std::to_string(i + 1) +
                " share no vertex",
            IBM_ERR_MESH);
        break;
      }
      v3 = (b0 == v2) ? b1 : b0;
      // the third edge must join v3 and v1
      if (!((c0 == v3 && c1 == v1) || (c0 == v1 && c1 == v3)) || v3 == v1) {
        bad("ibm_gts_read: the edges of face " + std::to_string(i + 1) + " do not form a triangle",
            IBM_ERR_MESH);
        break;
      }
      out.tri[3 * i] = (int32_t)v1;
      out.tri[3 * i + 1] = (int32_t)v2;
      out.tri[3 * i + 2] = (int32_t)v3;
    }
  }
  std::fclose(f);
  if (st != IBM_OK) return fail(msg, st);
  return IBM_OK;
}

}  // namespace

extern "C" ibm_status ibm_gts_read(const char* path, int64_t* n_vert, int64_t* n_face,
                                   double* xyz, int32_t* tri) {
  if (!path || !n_vert || !n_face) return fail("ibm_gts_read: null argument", IBM_ERR_INVALID_ARG);
  Gts g;
  const ibm_status st = parse(path, g);
  if (st != IBM_OK) return st;
  const int64_t nv = (int64_t)g.xyz.size() / 3, nf = (int64_t)g.tri.size() / 3;
  if (xyz || tri) {
    if (!xyz || !tri || *n_vert != nv || *n_face != nf)
      return fail("ibm_gts_read: buffers must be given together, sized by a first call",
                  IBM_ERR_INVALID_ARG);
    std::memcpy(xyz, g.xyz.data(), sizeof(double) * g.xyz.size());
    std::memcpy(tri, g.tri.data(), sizeof(int32_t) * g.tri.size());
  }
  *n_vert = nv;
  *n_face = nf;
  return IBM_OK;
}
