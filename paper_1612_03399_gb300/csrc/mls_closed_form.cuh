// Closed-form MLS shape functions of the factorised weight and their use on
// 3x3x3 supports (Sec. 2.2, Eqs. mls..mls_Q), shared by the marker kernels.
//
// MLS with the linear basis and a weight that factorises over directions
// (W = prod_d exp(-kappa delta_d^2), delta in cells) has an exact closed-form
// solution of the 4x4 moment system: with per-direction normalised weights
// a_d(s) = w_d(s)/S_d, mean mu_d and variance s2_d of the node offsets,
//   phi(sx,sy,sz) = a_x a_y a_z (1 - beta_x - beta_y - beta_z),
//   beta_d(s) = mu_d (delta_d(s) - mu_d) / s2_d.
// Writing b_d = a_d beta_d, phi = a_x a_y a_z - b_x a_y a_z - a_x b_y a_z
// - a_x a_y b_z, so value and full derivative are short tensor contractions of
// the 27 node values.
#pragma once

#include <cuda_runtime.h>
#include <limits.h>
#include <math.h>

#include "ibm_internal.cuh"

namespace ibm {
namespace {

struct DirW {
  float a[3], b[3];
};
struct DirWD {
  float a[3], b[3], da[3], db[3];
};

// per-direction closed-form MLS factors for the fractional offset tp in
// [-1/2, 1/2) of the point from its nearest node (cells).  The weights enter
// only through their ratios to the nearest node's,
//   w(-1)/w(0) = exp(-kappa (1 + 2 tp)),  w(+1)/w(0) = exp(-kappa (1 - 2 tp)),
// both in (0, 1], so two exponentials suffice and nothing overflows.
__device__ __forceinline__ void dir_weights(float tp, float kappa, DirW& o) {
  const float rm = __expf(-kappa * fmaf(2.f, tp, 1.f)), rp = __expf(-kappa * fmaf(-2.f, tp, 1.f));
  const float invS = __fdividef(1.f, 1.f + rm + rp);
  const float a0 = rm * invS, a1 = invS, a2 = rp * invS;
  const float d0 = -1.f - tp, d1 = -tp, d2 = 1.f - tp;
  const float mu = a0 * d0 + a1 * d1 + a2 * d2;
  const float e0 = d0 - mu, e1 = d1 - mu, e2 = d2 - mu;
  const float s2 = a0 * e0 * e0 + a1 * e1 * e1 + a2 * e2 * e2;
  const float r = __fdividef(mu, s2);
  o.a[0] = a0; o.a[1] = a1; o.a[2] = a2;
  o.b[0] = a0 * r * e0; o.b[1] = a1 * r * e1; o.b[2] = a2 * r * e2;
}

// the same factors and their derivatives with respect to the point's
// coordinate (in cells): the node offsets move as d delta / dt = -1, the
// weight ratios as d rm / dt = -2 kappa rm, d rp / dt = 2 kappa rp
__device__ __forceinline__ void dir_weights_d(float tp, float kappa, DirWD& o) {
  const float d[3] = {-1.f - tp, -tp, 1.f - tp};
  const float rm = __expf(-kappa * fmaf(2.f, tp, 1.f)), rp = __expf(-kappa * fmaf(-2.f, tp, 1.f));
  const float w[3] = {rm, 1.f, rp};
  const float dw[3] = {-2.f * kappa * rm, 0.f, 2.f * kappa * rp};
  const float invS = __fdividef(1.f, 1.f + rm + rp);
  const float dS = dw[0] + dw[2];
  float a[3], da[3];
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    a[s] = w[s] * invS;
    da[s] = (dw[s] - a[s] * dS) * invS;
  }
  const float mu = a[0] * d[0] + a[1] * d[1] + a[2] * d[2];
  const float dmu = da[0] * d[0] + da[1] * d[1] + da[2] * d[2] - 1.f;
  float e[3];
#pragma unroll
  for (int s = 0; s < 3; ++s) e[s] = d[s] - mu;
  const float s2 = a[0] * e[0] * e[0] + a[1] * e[1] * e[1] + a[2] * e[2] * e[2];
  const float ds2 = da[0] * e[0] * e[0] + da[1] * e[1] * e[1] + da[2] * e[2] * e[2];
  const float inv_s2 = __fdividef(1.f, s2);
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const float beta = mu * e[s] * inv_s2;
    const float dbeta = (dmu * e[s] + mu * (-1.f - dmu)) * inv_s2 - beta * ds2 * inv_s2;
    o.a[s] = a[s];
    o.b[s] = a[s] * beta;
    o.da[s] = da[s];
    o.db[s] = da[s] * beta + a[s] * dbeta;
  }
}

__device__ __forceinline__ int wrap(int i, int n) {
  if (i >= 0 && i < n) return i;
  if (i < 0 && i >= -n) return i + n;
  if (i >= n && i < 2 * n) return i - n;
  i %= n;
  return i < 0 ? i + n : i;
}

// Centre node (unwrapped global lattice index) and fractional offset of a
// point, in every direction, on the lattice of velocity component `comp`
// (node offset 0 along the component's own direction, 1/2 across it).
__device__ __forceinline__ void locate(const float (&tau)[3], int comp, const int (&G)[3],
                                       int (&c)[3], float (&tp)[3]) {
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float u = tau[d] - (d == comp ? 0.f : 0.5f);
    const float cc = floorf(u + 0.5f);
    tp[d] = u - cc;
    c[d] = G[d] + (int)cc;
  }
}

// addressing of a 3x3x3 support: rows (sy, sz), columns sx
struct GlobalAcc {   // wrapped indices into a full [nz][ny][nx] field
  int ix[3], iy[3], iz[3];
  int nx, ny;
  __device__ void init(const int (&c)[3], const Grid& g) {
    nx = g.n[0];
    ny = g.n[1];
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      ix[s] = wrap(c[0] - 1 + s, g.n[0]);
      iy[s] = wrap(c[1] - 1 + s, g.n[1]);
      iz[s] = wrap(c[2] - 1 + s, g.n[2]);
    }
  }
  __device__ int row(int sy, int sz) const { return (iz[sz] * ny + iy[sy]) * nx; }
  __device__ int col(int sx) const { return ix[sx]; }
};
struct RowAcc {      // indices into the rows staged in shared memory
  const int* off;    // staged offset of row r, minus its first x
  int ylo, zlo, sy;
  int cx, cy, cz;    // support corner (centre - 1)
  __device__ void init(const int (&c)[3], const int* off_minus_x0, int ylo_, int zlo_, int sy_) {
    off = off_minus_x0;
    ylo = ylo_;
    zlo = zlo_;
    sy = sy_;
    cx = c[0] - 1;
    cy = c[1] - 1;
    cz = c[2] - 1;
  }
  __device__ int row(int a, int b) const { return off[(cy + a - ylo) + sy * (cz + b - zlo)] + cx; }
  __device__ int col(int s) const { return s; }
};

// The contractions below run x first (per row, the a- and b-weighted sums as
// one pair in packed two-lane float arithmetic), then y within each z-plane,
// then z:  U = sum_z [a_z (P1 - P2 - P3) - b_z P1],  P1 = sum_y a_y xa,
// P2 = sum_y a_y xb, P3 = sum_y b_y xa.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

template <class Acc>
__device__ __forceinline__ float mls_value(const float* __restrict__ f, const Acc& A, const DirW& X,
                                           const DirW& Y, const DirW& Z) {
  const float2 ab0 = make_float2(X.a[0], X.b[0]), ab1 = make_float2(X.a[1], X.b[1]),
               ab2 = make_float2(X.a[2], X.b[2]);
  float q = 0.f;
#pragma unroll
  for (int sz = 0; sz < 3; ++sz) {
    float2 P = make_float2(0.f, 0.f);
    float P3 = 0.f;
#pragma unroll
    for (int sy = 0; sy < 3; ++sy) {
      const float* r = f + A.row(sy, sz);
      const float u0 = r[A.col(0)], u1 = r[A.col(1)], u2 = r[A.col(2)];
      float2 x2 = __ffma2_rn(ab0, f2(u0), make_float2(0.f, 0.f));
      x2 = __ffma2_rn(ab1, f2(u1), x2);
      x2 = __ffma2_rn(ab2, f2(u2), x2);
      P = __ffma2_rn(f2(Y.a[sy]), x2, P);
      P3 = fmaf(Y.b[sy], x2.x, P3);
    }
    q = fmaf(Z.a[sz], P.x - P.y - P3, fmaf(-Z.b[sz], P.x, q));
  }
  return q;
}

template <class Acc>
__device__ __forceinline__ void mls_grad(const float* __restrict__ f, const Acc& A, const DirWD& X,
                                         const DirWD& Y, const DirWD& Z, float (&g)[3]) {
  const float2 ab0 = make_float2(X.a[0], X.b[0]), ab1 = make_float2(X.a[1], X.b[1]),
               ab2 = make_float2(X.a[2], X.b[2]);
  const float2 db0 = make_float2(X.da[0], X.db[0]), db1 = make_float2(X.da[1], X.db[1]),
               db2 = make_float2(X.da[2], X.db[2]);
  float gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
  for (int sz = 0; sz < 3; ++sz) {
    // per plane: P = sum_y a_y (xa, xb), P3 = sum_y b_y xa; the same with the
    // x-derivative sums (Pd, Pd3) and with the y-derivative factors (Q, Q3)
    float2 P = make_float2(0.f, 0.f), Pd = P, Q = P;
    float P3 = 0.f, Pd3 = 0.f, Q3 = 0.f;
#pragma unroll
    for (int sy = 0; sy < 3; ++sy) {
      const float* r = f + A.row(sy, sz);
      const float u0 = r[A.col(0)], u1 = r[A.col(1)], u2 = r[A.col(2)];
      float2 x2 = __ffma2_rn(ab0, f2(u0), make_float2(0.f, 0.f));
      x2 = __ffma2_rn(ab1, f2(u1), x2);
      x2 = __ffma2_rn(ab2, f2(u2), x2);
      float2 d2 = __ffma2_rn(db0, f2(u0), make_float2(0.f, 0.f));
      d2 = __ffma2_rn(db1, f2(u1), d2);
      d2 = __ffma2_rn(db2, f2(u2), d2);
      P = __ffma2_rn(f2(Y.a[sy]), x2, P);
      P3 = fmaf(Y.b[sy], x2.x, P3);
      Pd = __ffma2_rn(f2(Y.a[sy]), d2, Pd);
      Pd3 = fmaf(Y.b[sy], d2.x, Pd3);
      Q = __ffma2_rn(f2(Y.da[sy]), x2, Q);
      Q3 = fmaf(Y.db[sy], x2.x, Q3);
    }
    gx = fmaf(Z.a[sz], Pd.x - Pd.y - Pd3, fmaf(-Z.b[sz], Pd.x, gx));
    gy = fmaf(Z.a[sz], Q.x - Q.y - Q3, fmaf(-Z.b[sz], Q.x, gy));
    gz = fmaf(Z.da[sz], P.x - P.y - P3, fmaf(-Z.db[sz], P.x, gz));
  }
  g[0] = gx; g[1] = gy; g[2] = gz;
}

// spread coef * phi onto the 27 nodes
template <class Acc>
__device__ __forceinline__ void mls_spread(float* f, const Acc& A, const DirW& X, const DirW& Y,
                                           const DirW& Z, float coef) {
#pragma unroll
  for (int sz = 0; sz < 3; ++sz) {
#pragma unroll
    for (int sy = 0; sy < 3; ++sy) {
      float* r = f + A.row(sy, sz);
      const float ay = Y.a[sy], by = Y.b[sy], az = Z.a[sz], bz = Z.b[sz];
      const float t0 = ay * az * coef, t1 = (by * az + ay * bz) * coef;
#pragma unroll
      for (int sx = 0; sx < 3; ++sx)
        atomicAdd(r + A.col(sx), (X.a[sx] - X.b[sx]) * t0 - X.a[sx] * t1);
    }
  }
}

// full-derivative MLS gradient (in cells) of component `comp` at a point
template <class Acc>
__device__ __forceinline__ void grad_at(const float* f, const Acc& A, const float (&tp)[3],
                                        float kappa, float (&gr)[3]) {
  DirWD X, Y, Z;
  dir_weights_d(tp[0], kappa, X);
  dir_weights_d(tp[1], kappa, Y);
  dir_weights_d(tp[2], kappa, Z);
  mls_grad(f, A, X, Y, Z, gr);
}

// x >= 0 folded into [0, n)
__device__ __forceinline__ int wrap_pos(int x, int n) {
  if (x >= n) {
    x -= n;
    if (x >= n) x %= n;
  }
  return x;
}

// asynchronous global -> shared copies (cp.async: no register round trip, so
// one thread's copies are all in flight at once)
__device__ __forceinline__ void cp_async16(float* sdst, const float* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async4(float* sdst, const float* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// the staged rows of the block, one float4 group (4 consecutive staged nodes
// of one row) per entry: the global offset of the group's first node
struct RowTable {
  const int* gofs;             // global offset of each group's first node
  int nx, vec4;
  // global offset of node j (0..3) of group q (without vector access a group
  // may cross the periodic x boundary: its nodes are wrapped one by one)
  __device__ __forceinline__ size_t node(int q, int j) const {
    const int g = gofs[q];
    if (vec4 || j == 0) return (size_t)g + j;
    const int x = g % nx;
    return (size_t)(g - x) + (x + j < nx ? x + j : x + j - nx);
  }
};

// issue the copies of one field component's staged rows into dst
__device__ __forceinline__ void stage_async(float* dst, const float* __restrict__ src,
                                            const RowTable& R, int ngroups) {
  for (int q = threadIdx.x; q < ngroups; q += blockDim.x) {
    if (R.vec4) {
      cp_async16(dst + 4 * q, src + R.node(q, 0));   // x multiple of 4 and nx % 4 == 0
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) cp_async4(dst + 4 * q + j, src + R.node(q, j));
    }
  }
}

// addressing factories: staged rows or the global field
struct StagedRows {
  const int* off_minus_x0;
  int ylo, zlo, sy;
  __device__ RowAcc at(const int (&c)[3]) const {
    RowAcc A;
    A.init(c, off_minus_x0, ylo, zlo, sy);
    return A;
  }
};
struct GlobalRows {
  Grid g;
  __device__ GlobalAcc at(const int (&c)[3]) const {
    GlobalAcc A;
    A.init(c, g);
    return A;
  }
};

// nearest node and derivative factors of one component at a probe point
struct ProbeW {
  int cc[3];
  DirWD X, Y, Z;
  __device__ __forceinline__ void prepare(const float (&t)[3], int comp, const int (&G)[3],
                                          float kappa) {
    float t3[3];
    locate(t, comp, G, cc, t3);
    dir_weights_d(t3[0], kappa, X);
    dir_weights_d(t3[1], kappa, Y);
    dir_weights_d(t3[2], kappa, Z);
  }
  // full-derivative gradient per unit length, times sgn, added to gr
  template <class Rows>
  __device__ __forceinline__ void add_gradient(const float* f, const Rows& R,
                                               const float (&invh)[3], float sgn,
                                               float (&gr)[3]) const {
    float gl[3];
    mls_grad(f, R.at(cc), X, Y, Z, gl);
#pragma unroll
    for (int j = 0; j < 3; ++j) gr[j] += sgn * gl[j] * invh[j];
  }
};

// bound on |phi| over the 27 nodes: phi = a_x a_y a_z - b_x a_y a_z - a_x b_y a_z
// - a_x a_y b_z, so |phi| <= prod_d (max|a_d| + max|b_d|)
__device__ __forceinline__ float phi_bound(const DirW& X, const DirW& Y, const DirW& Z) {
  auto p = [](const DirW& W) {
    return fmaxf(fmaxf(W.a[0], W.a[1]), W.a[2]) +
           fmaxf(fmaxf(fabsf(W.b[0]), fabsf(W.b[1])), fabsf(W.b[2]));
  };
  return p(X) * p(Y) * p(Z);
}

// Spread in exact fixed point: the contribution coef*phi, already scaled by
// the block's power of two so that |value| <= 2^38, is split into
// hi = floor(value / 2^16) (|hi| <= 2^22) and lo = value - 2^16 hi in
// [0, 2^16], each added with a native 32-bit shared atomic.  A node receives
// at most kMT contributions, so neither word overflows, and the node's sum
// 2^16 * sum(hi) + sum(lo) is independent of the order of the additions.
__device__ __forceinline__ void mls_spread_fixed(int* hi, int* lo, const RowAcc& A, const DirW& X,
                                                 const DirW& Y, const DirW& Z, float coef) {
#pragma unroll
  for (int sz = 0; sz < 3; ++sz) {
#pragma unroll
    for (int sy = 0; sy < 3; ++sy) {
      const int r = A.row(sy, sz);
      const float ay = Y.a[sy], by = Y.b[sy], az = Z.a[sz], bz = Z.b[sz];
      const float t0 = ay * az * coef, t1 = (by * az + ay * bz) * coef;
#pragma unroll
      for (int sx = 0; sx < 3; ++sx) {
        const float val = (X.a[sx] - X.b[sx]) * t0 - X.a[sx] * t1;
        const float hf = floorf(val * (1.f / 65536.f));
        atomicAdd(hi + r + sx, (int)hf);
        atomicAdd(lo + r + sx, __float2int_rn(fmaf(-hf, 65536.f, val)));
      }
    }
  }
}

// Spread in exact fixed point, one 32-bit word per node: the contribution
// coef*phi, already scaled by the block's power of two so that
// |value| < 2^22, rounded to an integer and added with a native shared
// atomic; a node receives at most kMT contributions, so the word does not
// overflow, and the sum is independent of the order of the additions.
__device__ __forceinline__ void mls_spread_fixed1(int* acc, const RowAcc& A, const DirW& X,
                                                  const DirW& Y, const DirW& Z, float coef) {
  // nodes 0 and 1 of each row in packed two-lane arithmetic
  const float2 d01 = make_float2(X.a[0] - X.b[0], X.a[1] - X.b[1]), a01 = make_float2(X.a[0], X.a[1]);
  const float d2 = X.a[2] - X.b[2];
#pragma unroll
  for (int sz = 0; sz < 3; ++sz) {
#pragma unroll
    for (int sy = 0; sy < 3; ++sy) {
      const int r = A.row(sy, sz);
      const float ay = Y.a[sy], by = Y.b[sy], az = Z.a[sz], bz = Z.b[sz];
      const float t0 = ay * az * coef, t1 = (by * az + ay * bz) * coef;
      const float2 v01 = __ffma2_rn(d01, f2(t0), __fmul2_rn(a01, f2(-t1)));
      atomicAdd(acc + r, __float2int_rn(v01.x));
      atomicAdd(acc + r + 1, __float2int_rn(v01.y));
      atomicAdd(acc + r + 2, __float2int_rn(fmaf(d2, t0, -X.a[2] * t1)));
    }
  }
}

// x (|x| < 2^62) rounded to a 64-bit integer without a 64-bit conversion:
// hi = floor(x / 2^32) is exact and the remainder x - 2^32 hi lies in [0, 2^32)
__device__ __forceinline__ long long to_fixed(float x) {
  const float hf = floorf(x * 0x1p-32f);
  const unsigned lo = __float2uint_rn(fmaf(-hf, 0x1p32f, x));
  return (long long)(int)hf * 4294967296ll + (long long)lo;
}

// 2^k as a float, k in [-126, 127]
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((k + 127) << 23); }

}  // namespace
}  // namespace ibm
