// Marker kernel: face geometry, per-body area/volume reductions, MLS
// interpolation at the centroid, direct-forcing marker force, probe gradient
// and traction, and spreading (Sec. 2.2, Eqs. mls..mls_cl; Sec. 5 steps 1-3).
//
// One block = up to kChunk faces (markers) of ONE body, one thread per face.
// Faces are ordered along a space-filling curve, so a block's markers form a
// compact surface patch.  The block first finds the grid box that holds every
// 3x3x3 support of its centroids and probe ends, stages u, v, w on that box in
// shared memory with coalesced row loads, interpolates from shared memory,
// accumulates its spread contributions in a shared force box with shared
// atomics, and flushes the box to the global force fields once (one global
// atomic per non-zero node instead of 81 per marker).  A block whose box does
// not fit falls back to direct global loads and atomics.
//
// MLS with the linear basis and a weight that factorises over directions
// (W = prod_d exp(-kappa delta_d^2), delta in cells) has an exact closed-form
// solution of the 4x4 moment system: with per-direction normalised weights
// a_d(s) = w_d(s)/S_d, mean mu_d and variance s2_d of the node offsets,
//   phi(sx,sy,sz) = a_x a_y a_z (1 - beta_x - beta_y - beta_z),
//   beta_d(s) = mu_d (delta_d(s) - mu_d) / s2_d.
// Writing b_d = a_d beta_d, phi = a_x a_y a_z - b_x a_y a_z - a_x b_y a_z
// - a_x a_y b_z, so value and full derivative are short tensor contractions of
// the 27 node values.  Partition of unity holds exactly, so c_l reduces to
// A_l (hx+hy+hz)/3 / (hx hy hz) on the uniform grid.
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
// [-1/2, 1/2) of the point from its nearest node (cells)
__device__ __forceinline__ void dir_weights(float tp, float kappa, DirW& o) {
  const float d0 = -1.f - tp, d1 = -tp, d2 = 1.f - tp;
  const float w0 = __expf(-kappa * d0 * d0), w1 = __expf(-kappa * d1 * d1),
              w2 = __expf(-kappa * d2 * d2);
  const float invS = 1.f / (w0 + w1 + w2);
  const float a0 = w0 * invS, a1 = w1 * invS, a2 = w2 * invS;
  const float mu = a0 * d0 + a1 * d1 + a2 * d2;
  const float e0 = d0 - mu, e1 = d1 - mu, e2 = d2 - mu;
  const float s2 = a0 * e0 * e0 + a1 * e1 * e1 + a2 * e2 * e2;
  const float r = mu / s2;
  o.a[0] = a0; o.a[1] = a1; o.a[2] = a2;
  o.b[0] = a0 * r * e0; o.b[1] = a1 * r * e1; o.b[2] = a2 * r * e2;
}

// the same factors and their derivatives with respect to the point's
// coordinate (in cells): the node offsets move as d delta / dt = -1
__device__ __forceinline__ void dir_weights_d(float tp, float kappa, DirWD& o) {
  float d[3] = {-1.f - tp, -tp, 1.f - tp};
  float w[3], dw[3];
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    w[s] = __expf(-kappa * d[s] * d[s]);
    dw[s] = w[s] * 2.f * kappa * d[s];
  }
  const float invS = 1.f / (w[0] + w[1] + w[2]);
  const float dS = dw[0] + dw[1] + dw[2];
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
  const float inv_s2 = 1.f / s2;
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

// addressing of the 3x3x3 support: rows (sy, sz) and columns sx
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
struct BoxAcc {      // indices into a box staged in shared memory
  int base, sx, sxy;
  __device__ void init(const int (&c)[3], const int (&lo)[3], const int (&s)[3]) {
    sx = s[0];
    sxy = s[0] * s[1];
    base = (c[0] - 1 - lo[0]) + sx * (c[1] - 1 - lo[1]) + sxy * (c[2] - 1 - lo[2]);
  }
  __device__ int row(int sy, int sz) const { return base + sz * sxy + sy * sx; }
  __device__ int col(int s) const { return s; }
};

template <class Acc>
__device__ __forceinline__ float mls_value(const float* __restrict__ f, const Acc& A, const DirW& X,
                                           const DirW& Y, const DirW& Z) {
  float q = 0.f;
#pragma unroll
  for (int sz = 0; sz < 3; ++sz) {
#pragma unroll
    for (int sy = 0; sy < 3; ++sy) {
      const float* r = f + A.row(sy, sz);
      const float u0 = r[A.col(0)], u1 = r[A.col(1)], u2 = r[A.col(2)];
      const float xa = X.a[0] * u0 + X.a[1] * u1 + X.a[2] * u2;
      const float xb = X.b[0] * u0 + X.b[1] * u1 + X.b[2] * u2;
      const float ay = Y.a[sy], by = Y.b[sy], az = Z.a[sz], bz = Z.b[sz];
      q += (xa - xb) * ay * az - xa * (by * az + ay * bz);
    }
  }
  return q;
}

template <class Acc>
__device__ __forceinline__ void mls_grad(const float* __restrict__ f, const Acc& A, const DirWD& X,
                                         const DirWD& Y, const DirWD& Z, float (&g)[3]) {
  float gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
  for (int sz = 0; sz < 3; ++sz) {
#pragma unroll
    for (int sy = 0; sy < 3; ++sy) {
      const float* r = f + A.row(sy, sz);
      const float u0 = r[A.col(0)], u1 = r[A.col(1)], u2 = r[A.col(2)];
      const float xa = X.a[0] * u0 + X.a[1] * u1 + X.a[2] * u2;
      const float xb = X.b[0] * u0 + X.b[1] * u1 + X.b[2] * u2;
      const float xda = X.da[0] * u0 + X.da[1] * u1 + X.da[2] * u2;
      const float xdb = X.db[0] * u0 + X.db[1] * u1 + X.db[2] * u2;
      const float ay = Y.a[sy], by = Y.b[sy], az = Z.a[sz], bz = Z.b[sz];
      const float day = Y.da[sy], dby = Y.db[sy], daz = Z.da[sz], dbz = Z.db[sz];
      gx += (xda - xdb) * ay * az - xda * (by * az + ay * bz);
      gy += (xa - xb) * day * az - xa * (dby * az + day * bz);
      gz += (xa - xb) * ay * daz - xa * (by * daz + ay * dbz);
    }
  }
  g[0] = gx; g[1] = gy; g[2] = gz;
}

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
      for (int sx = 0; sx < 3; ++sx) atomicAdd(r + A.col(sx), (X.a[sx] - X.b[sx]) * t0 - X.a[sx] * t1);
    }
  }
}

__device__ __forceinline__ void dir3(const float (&tp)[3], float kappa, DirW& X, DirW& Y, DirW& Z) {
  dir_weights(tp[0], kappa, X);
  dir_weights(tp[1], kappa, Y);
  dir_weights(tp[2], kappa, Z);
}

// full-derivative MLS gradient (in cells) of component `comp` at a point,
// from the staged box (box = true) or the global field
__device__ __forceinline__ void probe_gradient(const float* f, bool box, const float (&tau)[3],
                                               int comp, const BodyDev& B, const Grid& g,
                                               float kappa, const int (&lo)[3], const int (&sz)[3],
                                               float (&gr)[3]) {
  int c[3];
  float tp[3];
  locate(tau, comp, B.G, c, tp);
  DirWD X, Y, Z;
  dir_weights_d(tp[0], kappa, X);
  dir_weights_d(tp[1], kappa, Y);
  dir_weights_d(tp[2], kappa, Z);
  if (box) {
    BoxAcc A;
    A.init(c, lo, sz);
    mls_grad(f, A, X, Y, Z, gr);
  } else {
    GlobalAcc A;
    A.init(c, g);
    mls_grad(f, A, X, Y, Z, gr);
  }
}

// global offset of node r (x fastest) of the box with corner lo and size sz
__device__ __forceinline__ size_t box_node(int r, const int (&lo)[3], const int (&sz)[3], int sxy,
                                           const Grid& g) {
  const int k = r / sxy, rem = r - k * sxy, j = rem / sz[0], i = rem - j * sz[0];
  return ((size_t)wrap(lo[2] + k, g.n[2]) * g.n[1] + wrap(lo[1] + j, g.n[1])) * g.n[0] +
         wrap(lo[0] + i, g.n[0]);
}

// extend [lo, hi] by the supports of all three components at a point, with
// exactly the centre nodes the evaluation will use
__device__ __forceinline__ void minmax_loc(const float (&tau)[3], const int (&G)[3], int (&lo)[3],
                                           int (&hi)[3]) {
#pragma unroll
  for (int comp = 0; comp < 3; ++comp) {
    int c[3];
    float tp[3];
    locate(tau, comp, G, c, tp);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      lo[d] = min(lo[d], c[d] - 1);
      hi[d] = max(hi[d], c[d] + 1);
    }
  }
}

template <bool MEASURE, bool INTERP, bool PROBE, bool SPREAD>
__global__ void __launch_bounds__(kChunk, 4) marker_kernel(
    DeviceTables T, Grid g, StepConsts sc, int32_t V, int32_t F, const float* __restrict__ x,
    const float* __restrict__ v, const float* __restrict__ u, const float* __restrict__ vv,
    const float* __restrict__ w, float* __restrict__ U, float* __restrict__ Fm,
    const float* __restrict__ Fm_in, float* __restrict__ Fext, float* __restrict__ fx,
    float* __restrict__ fy, float* __restrict__ fz, int record_box) {
  constexpr bool FIELD = INTERP || PROBE || SPREAD;
  constexpr bool VEL = INTERP || PROBE;
  extern __shared__ float sbox[];
  __shared__ int s_lo[3], s_hi[3];
  __shared__ double s_red[2][kChunk / 32];
  __shared__ int s_last;
  __shared__ uint32_t s_mask[SPREAD ? kMaskWords : 1];
  const int4 ch = T.chunks[blockIdx.x];  // body, first local face, count, chunk index in body
  const BodyDev B = T.body[ch.x];
  const int tri_off = T.topo[B.topo].tri_off;
  const int lf = ch.y + threadIdx.x;
  const bool active = threadIdx.x < ch.z;
  if (FIELD && threadIdx.x < 3) {
    s_lo[threadIdx.x] = INT_MAX;
    s_hi[threadIdx.x] = INT_MIN;
  }
  float Af = 0.f, Vf = 0.f;
  float c[3] = {0.f, 0.f, 0.f}, nrm[3] = {0.f, 0.f, 0.f}, area = 0.f;
  float tc[3], tp[3], tm[3];
  bool ok = false;
  int ia = 0, ib = 0, ic = 0, gf = 0;
  if (active) {
    gf = B.f_off + lf;
    const int* tr = T.tri + tri_off + 3 * lf;
    ia = B.v_off + __ldg(tr);
    ib = B.v_off + __ldg(tr + 1);
    ic = B.v_off + __ldg(tr + 2);
    float xa[3], xb[3], xc[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      xa[d] = __ldg(x + d * V + ia);
      xb[d] = __ldg(x + d * V + ib);
      xc[d] = __ldg(x + d * V + ic);
    }
    const float e1[3] = {xb[0] - xa[0], xb[1] - xa[1], xb[2] - xa[2]};
    const float e2[3] = {xc[0] - xa[0], xc[1] - xa[1], xc[2] - xa[2]};
    const float N[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                        e1[0] * e2[1] - e1[1] * e2[0]};
    const float nn = sqrtf(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
    area = 0.5f * nn;
    if (MEASURE) {
      Af = area;
      if (B.closed) {
        Vf = (xa[0] * (xb[1] * xc[2] - xb[2] * xc[1]) + xa[1] * (xb[2] * xc[0] - xb[0] * xc[2]) +
              xa[2] * (xb[0] * xc[1] - xb[1] * xc[0])) * (1.f / 6.f);
      }
    }
    if (FIELD) {
      const float third = 1.f / 3.f;
      const float inv = 1.f / nn;
      ok = nn > 0.f;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        c[d] = (xa[d] + xb[d] + xc[d]) * third;
        nrm[d] = N[d] * inv;
        tc[d] = fmaf(c[d], g.invh[d], B.frac[d]);
        tp[d] = fmaf(c[d] + sc.probe_h * nrm[d], g.invh[d], B.frac[d]);
        tm[d] = fmaf(c[d] - sc.probe_h * nrm[d], g.invh[d], B.frac[d]);
        ok = ok && fabsf(tc[d]) < 1.0e7f && fabsf(tp[d]) < 1.0e7f && fabsf(tm[d]) < 1.0e7f;
      }
      if (!ok) atomicOr(T.err, ERR_NONFINITE);
    }
  }

  // ---- the block's grid box --------------------------------------------
  int lo[3] = {0, 0, 0}, sz[3] = {0, 0, 0};
  bool fit = false;
  int N = 0;
  if (FIELD) {
    int mlo[3] = {INT_MAX, INT_MAX, INT_MAX}, mhi[3] = {INT_MIN, INT_MIN, INT_MIN};
    if (active && ok) {
      minmax_loc(tc, B.G, mlo, mhi);
      if (PROBE) {
        minmax_loc(tp, B.G, mlo, mhi);
        if (!B.closed) minmax_loc(tm, B.G, mlo, mhi);
      }
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        mlo[d] = min(mlo[d], __shfl_xor_sync(0xffffffffu, mlo[d], o));
        mhi[d] = max(mhi[d], __shfl_xor_sync(0xffffffffu, mhi[d], o));
      }
    }
    if (SPREAD && record_box)
      for (int k = threadIdx.x; k < kMaskWords; k += blockDim.x) s_mask[k] = 0u;
    __syncthreads();   // s_lo / s_hi initialised
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        atomicMin(&s_lo[d], mlo[d]);
        atomicMax(&s_hi[d], mhi[d]);
      }
    }
    __syncthreads();
    long long nbox = 1;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      lo[d] = s_lo[d];
      sz[d] = s_hi[d] >= s_lo[d] ? s_hi[d] - s_lo[d] + 1 : 0;
      nbox *= sz[d];
    }
    // one velocity component (and its force component) is staged at a time
    const int nfield = (VEL ? 1 : 0) + (SPREAD ? 1 : 0);
    fit = nbox > 0 && nbox <= kMaxBoxNodes &&
          nbox * nfield * (long long)sizeof(float) <= kMarkerSmemBytes;
    N = fit ? (int)nbox : 0;
    if (!fit && nbox > 0 && threadIdx.x == 0) atomicAdd(T.stats, 1);
  }
  float* vbox = sbox;
  float* fbox = sbox + (VEL ? N : 0);
  const bool mine = FIELD && active && ok;

  // ---- per component: stage, interpolate, spread, differentiate, flush ----
  // Each component's interpolation, spreading and gradient use only that
  // component's field, so the shared box holds one component at a time.
  float G[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
  if (FIELD) {
    const int sxy = sz[0] * sz[1];
    const float third = 1.f / 3.f;
    const float cl = area * sc.cl_scale;
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
      const float* velc = comp == 0 ? u : (comp == 1 ? vv : w);
      float* frcc = comp == 0 ? fx : (comp == 1 ? fy : fz);
      if (fit) {
        __syncthreads();   // the previous component is done with the boxes
        for (int r = threadIdx.x; r < N; r += blockDim.x) {
          if (VEL) vbox[r] = __ldg(velc + box_node(r, lo, sz, sxy, g));
          if (SPREAD) fbox[r] = 0.f;
        }
        __syncthreads();
      }
      if (mine) {
        if (INTERP || SPREAD) {
          int cc[3];
          float t3[3];
          locate(tc, comp, B.G, cc, t3);
          DirW X, Y, Z;
          dir3(t3, sc.kappa, X, Y, Z);
          float Fl;
          if (INTERP) {
            float Ul;
            if (fit) {
              BoxAcc A;
              A.init(cc, lo, sz);
              Ul = mls_value(vbox, A, X, Y, Z);
            } else {
              GlobalAcc A;
              A.init(cc, g);
              Ul = mls_value(velc, A, X, Y, Z);
            }
            const float vb = (__ldg(v + comp * V + ia) + __ldg(v + comp * V + ib) +
                              __ldg(v + comp * V + ic)) * third;
            Fl = (vb - Ul) * sc.inv_dt;
            if (U) U[comp * F + gf] = Ul;
            if (Fm) Fm[comp * F + gf] = Fl;
          } else {
            Fl = __ldg(Fm_in + comp * F + gf);
          }
          if (SPREAD) {
            if (fit) {
              BoxAcc A;
              A.init(cc, lo, sz);
              mls_spread(fbox, A, X, Y, Z, cl * Fl);
            } else {
              GlobalAcc A;
              A.init(cc, g);
              mls_spread(frcc, A, X, Y, Z, cl * Fl);
            }
          }
        }
        if (PROBE) {
          float gr[3];
          probe_gradient(fit ? (const float*)vbox : velc, fit, tp, comp, B, g, sc.kappa, lo, sz, gr);
          if (!B.closed) {
            // open sheet: second probe on the other side, (tau+ - tau-) . n+
            float gm[3];
            probe_gradient(fit ? (const float*)vbox : velc, fit, tm, comp, B, g, sc.kappa, lo, sz,
                           gm);
#pragma unroll
            for (int j = 0; j < 3; ++j) gr[j] -= gm[j];
          }
#pragma unroll
          for (int j = 0; j < 3; ++j) G[comp][j] = gr[j] * g.invh[j];
        }
      }
      if (SPREAD && fit) {
        __syncthreads();
        for (int r = threadIdx.x; r < N; r += blockDim.x) {
          const float val = fbox[r];
          if (val != 0.f) {
            atomicAdd(frcc + box_node(r, lo, sz, sxy, g), val);
            if (record_box) atomicOr(&s_mask[r >> 5], 1u << (r & 31));
          }
        }
      }
    }
    if (PROBE && mine) {
      const float s = sc.mu * area;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const float t = (G[i][0] + G[0][i]) * nrm[0] + (G[i][1] + G[1][i]) * nrm[1] +
                        (G[i][2] + G[2][i]) * nrm[2];
        Fext[i * F + gf] = s * t;
      }
    }
    if (SPREAD && record_box) {
      // footprint for the next step's clear: exact node mask when the box was
      // staged, the whole box (flag 1) otherwise; a box wider than the grid
      // covers that whole direction
      __syncthreads();
      const int gc = B.chunk_off + ch.w;
      if (fit)
        for (int k = threadIdx.x; k < (N + 31) / 32; k += blockDim.x)
          T.mask[(size_t)gc * kMaskWords + k] = s_mask[k];
      if (threadIdx.x == 0) {
        T.boxes[2 * gc] = make_int4(lo[0], lo[1], lo[2], fit ? 0 : 1);
        T.boxes[2 * gc + 1] =
            make_int4(min(sz[0], g.n[0]), min(sz[1], g.n[1]), min(sz[2], g.n[2]), 0);
      }
    }
  }

  // ---- per-body float64 area and volume ------------------------------------
  if (MEASURE) {
    // fixed-order reduction: warp shuffles, warps in order, one partial per
    // chunk; the last chunk of the body to arrive sums the partials in order
    double a = (double)Af, vol = (double)Vf;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      vol += __shfl_down_sync(0xffffffffu, vol, o);
    }
    if ((threadIdx.x & 31) == 0) {
      s_red[0][threadIdx.x >> 5] = a;
      s_red[1][threadIdx.x >> 5] = vol;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double sa = 0.0, sv = 0.0;
      for (int k = 0; k < kChunk / 32; ++k) {
        sa += s_red[0][k];
        sv += s_red[1][k];
      }
      const int gc = B.chunk_off + ch.w;
      T.partial[2 * gc] = sa;
      T.partial[2 * gc + 1] = sv;
      __threadfence();
      const int arrived = atomicAdd(T.counter + ch.x, 1);
      s_last = (arrived == B.n_chunk - 1);
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
      __threadfence();
      double ta = 0.0, tv = 0.0;
      const volatile double* P = T.partial;
      for (int k = 0; k < B.n_chunk; ++k) {
        ta += P[2 * (B.chunk_off + k)];
        tv += P[2 * (B.chunk_off + k) + 1];
      }
      T.meas[2 * ch.x] = ta;
      T.meas[2 * ch.x + 1] = tv;
      const float cA = (float)(B.kA * ((ta - B.A0) / B.A0));
      const float cV = B.closed ? (float)(B.kv * ((tv - B.V0) / B.V0)) : 0.f;
      T.coef[ch.x] = make_float2(cA, cV);
      T.counter[ch.x] = 0;
    }
  }
}

// zero the three force fields on every box recorded by the previous spread
__global__ void __launch_bounds__(256) clear_kernel(DeviceTables T, Grid g, float* __restrict__ fx,
                                                    float* __restrict__ fy, float* __restrict__ fz) {
  const int4 lo = T.boxes[2 * blockIdx.x];
  const int4 sz = T.boxes[2 * blockIdx.x + 1];
  const long long N = (long long)sz.x * sz.y * sz.z;
  if (N <= 0) return;
  const int sxy = sz.x * sz.y;
  const bool whole = lo.w != 0;
  const uint32_t* mask = T.mask + (size_t)blockIdx.x * kMaskWords;
  for (long long idx = threadIdx.x; idx < N; idx += blockDim.x) {
    if (!whole && !((__ldg(mask + (idx >> 5)) >> (idx & 31)) & 1u)) continue;
    const int k = (int)(idx / sxy), rem = (int)(idx - (long long)k * sxy), j = rem / sz.x,
              i = rem - j * sz.x;
    const size_t o = ((size_t)wrap(lo.z + k, g.n[2]) * g.n[1] + wrap(lo.y + j, g.n[1])) * g.n[0] +
                     wrap(lo.x + i, g.n[0]);
    fx[o] = 0.f;
    fy[o] = 0.f;
    fz[o] = 0.f;
  }
  __syncthreads();
  if (threadIdx.x == 0) T.boxes[2 * blockIdx.x + 1] = make_int4(0, 0, 0, 0);
}

template <bool M, bool I, bool P, bool S>
cudaError_t launch_t(ibm_ctx* c, const float* x, const float* v, const float* u, const float* vv,
                     const float* w, float* U, float* Fm, const float* Fm_in, float* Fext,
                     float* fx, float* fy, float* fz, int record_box) {
  if (c->n_chunks == 0) return cudaSuccess;
  const size_t smem = (I || P || S) ? kMarkerSmemBytes : 0;
  marker_kernel<M, I, P, S><<<c->n_chunks, kChunk, smem, c->stream>>>(
      c->d, c->grid, c->sc, (int32_t)c->V, (int32_t)c->F, x, v, u, vv, w, U, Fm, Fm_in, Fext,
      fx, fy, fz, record_box);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_mls(ibm_ctx* c, const float* x, const float* v, const float* u,
                       const float* vv, const float* w, float* U, float* Fm, const float* Fm_in,
                       float* Fext, float* fx, float* fy, float* fz, bool measure, bool interp,
                       bool probe, bool spread, bool record_box) {
  const int rb = record_box ? 1 : 0;
  if (measure && interp && probe && spread)
    return launch_t<true, true, true, true>(c, x, v, u, vv, w, U, Fm, Fm_in, Fext, fx, fy, fz, rb);
  if (measure && !interp && !probe && !spread)
    return launch_t<true, false, false, false>(c, x, v, u, vv, w, U, Fm, Fm_in, Fext, fx, fy, fz, rb);
  if (!measure && interp && probe && !spread)
    return launch_t<false, true, true, false>(c, x, v, u, vv, w, U, Fm, Fm_in, Fext, fx, fy, fz, rb);
  if (!measure && interp && !probe && !spread)
    return launch_t<false, true, false, false>(c, x, v, u, vv, w, U, Fm, Fm_in, Fext, fx, fy, fz, rb);
  if (!measure && !interp && probe && !spread)
    return launch_t<false, false, true, false>(c, x, v, u, vv, w, U, Fm, Fm_in, Fext, fx, fy, fz, rb);
  if (!measure && !interp && !probe && spread)
    return launch_t<false, false, false, true>(c, x, v, u, vv, w, U, Fm, Fm_in, Fext, fx, fy, fz, rb);
  return cudaErrorInvalidValue;
}

cudaError_t launch_clear(ibm_ctx* c, float* fx, float* fy, float* fz) {
  if (c->n_chunks == 0) return cudaSuccess;
  clear_kernel<<<c->n_chunks, 256, 0, c->stream>>>(c->d, c->grid, fx, fy, fz);
  return cudaGetLastError();
}

}  // namespace ibm
