// Marker kernels: face geometry, per-body area/volume reductions, MLS
// interpolation at the centroid, direct-forcing marker force, probe gradient
// and traction, and spreading (Sec. 2.2, Eqs. mls..mls_cl; Sec. 5 steps 1-3).
//
// One thread per face (marker).  A block holds up to kChunk faces of ONE body,
// so every body scalar is uniform across the block.
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

// three wrapped node indices ic-1, ic, ic+1 of one direction
__device__ __forceinline__ void node3(int c, int n, int (&o)[3]) {
  const int m = wrap(c - 1, n);
  o[0] = m;
  o[1] = (m + 1 == n) ? 0 : m + 1;
  o[2] = (o[1] + 1 == n) ? 0 : o[1] + 1;
}

// Location of a point in one direction for a lattice with node offset `off`
// (0 or 1/2 cell): tau = position / h in cells relative to the body's
// integer origin G; returns the centre node (global, unwrapped) and the
// fractional offset.
__device__ __forceinline__ int locate(float tau, float off, int G, float& tp) {
  const float u = tau - off;
  const float c = floorf(u + 0.5f);
  tp = u - c;
  return G + (int)c;
}

// value of the MLS interpolant of `f` (one component) at the point
__device__ __forceinline__ float mls_value(const float* __restrict__ f, const int (&ix)[3],
                                           const int (&iy)[3], const int (&iz)[3], int nx,
                                           int ny, const DirW& X, const DirW& Y,
                                           const DirW& Z) {
  float q = 0.f;
#pragma unroll
  for (int sz = 0; sz < 3; ++sz) {
#pragma unroll
    for (int sy = 0; sy < 3; ++sy) {
      const int base = (iz[sz] * ny + iy[sy]) * nx;
      const float u0 = __ldg(f + base + ix[0]), u1 = __ldg(f + base + ix[1]),
                  u2 = __ldg(f + base + ix[2]);
      const float xa = X.a[0] * u0 + X.a[1] * u1 + X.a[2] * u2;
      const float xb = X.b[0] * u0 + X.b[1] * u1 + X.b[2] * u2;
      const float ay = Y.a[sy], by = Y.b[sy], az = Z.a[sz], bz = Z.b[sz];
      q += (xa - xb) * ay * az - xa * (by * az + ay * bz);
    }
  }
  return q;
}

// full derivative (in cells) of the MLS interpolant at the point
__device__ __forceinline__ void mls_grad(const float* __restrict__ f, const int (&ix)[3],
                                         const int (&iy)[3], const int (&iz)[3], int nx, int ny,
                                         const DirWD& X, const DirWD& Y, const DirWD& Z,
                                         float (&g)[3]) {
  float gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
  for (int sz = 0; sz < 3; ++sz) {
#pragma unroll
    for (int sy = 0; sy < 3; ++sy) {
      const int base = (iz[sz] * ny + iy[sy]) * nx;
      const float u0 = __ldg(f + base + ix[0]), u1 = __ldg(f + base + ix[1]),
                  u2 = __ldg(f + base + ix[2]);
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

__device__ __forceinline__ void mls_spread(float* __restrict__ f, const int (&ix)[3],
                                           const int (&iy)[3], const int (&iz)[3], int nx,
                                           int ny, const DirW& X, const DirW& Y, const DirW& Z,
                                           float coef) {
#pragma unroll
  for (int sz = 0; sz < 3; ++sz) {
#pragma unroll
    for (int sy = 0; sy < 3; ++sy) {
      const int base = (iz[sz] * ny + iy[sy]) * nx;
      const float ay = Y.a[sy], by = Y.b[sy], az = Z.a[sz], bz = Z.b[sz];
      const float t0 = ay * az * coef, t1 = (by * az + ay * bz) * coef;
#pragma unroll
      for (int sx = 0; sx < 3; ++sx) {
        const float phi_c = (X.a[sx] - X.b[sx]) * t0 - X.a[sx] * t1;
        atomicAdd(f + base + ix[sx], phi_c);
      }
    }
  }
}

// gradient tensor G[i][j] = d u_i / d x_j of the three staggered components
// at body-frame point p
__device__ __forceinline__ void velocity_gradient(const float* __restrict__ u,
                                                  const float* __restrict__ vv,
                                                  const float* __restrict__ w, const Grid& g,
                                                  const BodyDev& B, float kappa, const float (&p)[3],
                                                  float (&G)[3][3]) {
  float tau[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) tau[d] = fmaf(p[d], g.invh[d], B.frac[d]);
  // direction factors for node offset 0 (index 0) and 1/2 (index 1)
  DirWD W0[3], W1[3];
  int I0[3][3], I1[3][3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    float tp;
    int c = locate(tau[d], 0.f, B.G[d], tp);
    dir_weights_d(tp, kappa, W0[d]);
    node3(c, g.n[d], I0[d]);
    c = locate(tau[d], 0.5f, B.G[d], tp);
    dir_weights_d(tp, kappa, W1[d]);
    node3(c, g.n[d], I1[d]);
  }
  float gr[3];
  mls_grad(u, I0[0], I1[1], I1[2], g.n[0], g.n[1], W0[0], W1[1], W1[2], gr);
#pragma unroll
  for (int j = 0; j < 3; ++j) G[0][j] = gr[j] * g.invh[j];
  mls_grad(vv, I1[0], I0[1], I1[2], g.n[0], g.n[1], W1[0], W0[1], W1[2], gr);
#pragma unroll
  for (int j = 0; j < 3; ++j) G[1][j] = gr[j] * g.invh[j];
  mls_grad(w, I1[0], I1[1], I0[2], g.n[0], g.n[1], W1[0], W1[1], W0[2], gr);
#pragma unroll
  for (int j = 0; j < 3; ++j) G[2][j] = gr[j] * g.invh[j];
}

template <bool MEASURE, bool INTERP, bool PROBE, bool SPREAD>
__global__ void __launch_bounds__(kChunk) marker_kernel(
    DeviceTables T, Grid g, StepConsts sc, int32_t V, int32_t F, const float* __restrict__ x,
    const float* __restrict__ v, const float* __restrict__ u, const float* __restrict__ vv,
    const float* __restrict__ w, float* __restrict__ U, float* __restrict__ Fm,
    const float* __restrict__ Fm_in, float* __restrict__ Fext, float* __restrict__ fx,
    float* __restrict__ fy, float* __restrict__ fz, uint8_t* __restrict__ bricks,
    int3 nbrick) {
  const int4 ch = T.chunks[blockIdx.x];  // body, first local face, count, chunk index
  const BodyDev B = T.body[ch.x];
  const TopoDev topo = T.topo[B.topo];
  const int lf = ch.y + threadIdx.x;
  const bool active = threadIdx.x < ch.z;
  double Af = 0.0, Vf = 0.0;
  if (active) {
    const int gf = B.f_off + lf;
    const int* tr = T.tri + topo.tri_off + 3 * lf;
    const int ia = B.v_off + __ldg(tr), ib = B.v_off + __ldg(tr + 1), ic = B.v_off + __ldg(tr + 2);
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
    const float area = 0.5f * nn;
    if (MEASURE) {
      Af = (double)area;
      if (B.closed) {
        const float cbc[3] = {xb[1] * xc[2] - xb[2] * xc[1], xb[2] * xc[0] - xb[0] * xc[2],
                              xb[0] * xc[1] - xb[1] * xc[0]};
        Vf = (double)(xa[0] * cbc[0] + xa[1] * cbc[1] + xa[2] * cbc[2]) * (1.0 / 6.0);
      }
    }
    if (INTERP || PROBE || SPREAD) {
      const float third = 1.f / 3.f;
      const float c[3] = {(xa[0] + xb[0] + xc[0]) * third, (xa[1] + xb[1] + xc[1]) * third,
                          (xa[2] + xb[2] + xc[2]) * third};
      float tau[3];
      bool ok = nn > 0.f;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        tau[d] = fmaf(c[d], g.invh[d], B.frac[d]);
        ok = ok && fabsf(tau[d]) < 1.0e7f;   // also false for NaN
      }
      if (!ok) {
        atomicOr(T.err, ERR_NONFINITE);
      } else {
        if (INTERP || SPREAD) {
          DirW W0[3], W1[3];
          int I0[3][3], I1[3][3];
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            float tp;
            int cc = locate(tau[d], 0.f, B.G[d], tp);
            dir_weights(tp, sc.kappa, W0[d]);
            node3(cc, g.n[d], I0[d]);
            cc = locate(tau[d], 0.5f, B.G[d], tp);
            dir_weights(tp, sc.kappa, W1[d]);
            node3(cc, g.n[d], I1[d]);
          }
          float Fl[3];
          if (INTERP) {
            float Ul[3];
            Ul[0] = mls_value(u, I0[0], I1[1], I1[2], g.n[0], g.n[1], W0[0], W1[1], W1[2]);
            Ul[1] = mls_value(vv, I1[0], I0[1], I1[2], g.n[0], g.n[1], W1[0], W0[1], W1[2]);
            Ul[2] = mls_value(w, I1[0], I1[1], I0[2], g.n[0], g.n[1], W1[0], W1[1], W0[2]);
#pragma unroll
            for (int d = 0; d < 3; ++d) {
              const float vb = (__ldg(v + d * V + ia) + __ldg(v + d * V + ib) +
                                __ldg(v + d * V + ic)) * third;
              Fl[d] = (vb - Ul[d]) * sc.inv_dt;
            }
            if (U) {
#pragma unroll
              for (int d = 0; d < 3; ++d) U[d * F + gf] = Ul[d];
            }
            if (Fm) {
#pragma unroll
              for (int d = 0; d < 3; ++d) Fm[d * F + gf] = Fl[d];
            }
          } else {
#pragma unroll
            for (int d = 0; d < 3; ++d) Fl[d] = __ldg(Fm_in + d * F + gf);
          }
          if (SPREAD) {
            const float cl = area * sc.cl_scale;
            mls_spread(fx, I0[0], I1[1], I1[2], g.n[0], g.n[1], W0[0], W1[1], W1[2], cl * Fl[0]);
            mls_spread(fy, I1[0], I0[1], I1[2], g.n[0], g.n[1], W1[0], W0[1], W1[2], cl * Fl[1]);
            mls_spread(fz, I1[0], I1[1], I0[2], g.n[0], g.n[1], W1[0], W1[1], W0[2], cl * Fl[2]);
            if (bricks) {
              // mark the 8^3-cell bricks overlapped by the footprint (cells
              // floor(tau)-1 .. floor(tau)+2 hold every component's stencil)
              int lo[3], hi[3];
#pragma unroll
              for (int d = 0; d < 3; ++d) {
                const int c0 = B.G[d] + (int)floorf(tau[d]);
                lo[d] = wrap(c0 - 1, g.n[d]) >> 3;
                hi[d] = wrap(c0 + 2, g.n[d]) >> 3;
              }
              const int bx[2] = {lo[0], hi[0]}, by[2] = {lo[1], hi[1]}, bz[2] = {lo[2], hi[2]};
#pragma unroll
              for (int k = 0; k < 2; ++k)
#pragma unroll
                for (int j = 0; j < 2; ++j)
#pragma unroll
                  for (int i = 0; i < 2; ++i)
                    bricks[(bz[k] * nbrick.y + by[j]) * nbrick.x + bx[i]] = 1;
            }
          }
        }
        if (PROBE) {
          const float inv = 1.f / nn;
          const float n[3] = {N[0] * inv, N[1] * inv, N[2] * inv};
          const float p[3] = {c[0] + sc.probe_h * n[0], c[1] + sc.probe_h * n[1],
                              c[2] + sc.probe_h * n[2]};
          float G[3][3];
          velocity_gradient(u, vv, w, g, B, sc.kappa, p, G);
          if (!B.closed) {
            // open sheet: second probe on the other side, (tau+ - tau-) . n+
            const float pm[3] = {c[0] - sc.probe_h * n[0], c[1] - sc.probe_h * n[1],
                                 c[2] - sc.probe_h * n[2]};
            float Gm[3][3];
            velocity_gradient(u, vv, w, g, B, sc.kappa, pm, Gm);
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
              for (int j = 0; j < 3; ++j) G[i][j] -= Gm[i][j];
          }
          const float s = sc.mu * area;
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            const float t = (G[i][0] + G[0][i]) * n[0] + (G[i][1] + G[1][i]) * n[1] +
                            (G[i][2] + G[2][i]) * n[2];
            Fext[i * F + gf] = s * t;
          }
        }
      }
    }
  }
  if (MEASURE) {
    // deterministic per-body float64 sums: fixed-order block reduction, one
    // partial per chunk, and the last chunk of the body to arrive adds the
    // partials in chunk order
    __shared__ double sA[kChunk], sV[kChunk];
    __shared__ int last;
    sA[threadIdx.x] = Af;
    sV[threadIdx.x] = Vf;
    __syncthreads();
#pragma unroll
    for (int s = kChunk / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) {
        sA[threadIdx.x] += sA[threadIdx.x + s];
        sV[threadIdx.x] += sV[threadIdx.x + s];
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      const int gc = B.chunk_off + ch.w;
      T.partial[2 * gc] = sA[0];
      T.partial[2 * gc + 1] = sV[0];
      __threadfence();
      const int arrived = atomicAdd(T.counter + ch.x, 1);
      last = (arrived == B.n_chunk - 1);
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
      __threadfence();
      double a = 0.0, vol = 0.0;
      const volatile double* P = T.partial;
      for (int k = 0; k < B.n_chunk; ++k) {
        a += P[2 * (B.chunk_off + k)];
        vol += P[2 * (B.chunk_off + k) + 1];
      }
      T.meas[2 * ch.x] = a;
      T.meas[2 * ch.x + 1] = vol;
      T.counter[ch.x] = 0;
    }
  }
}

// zero the three force fields on every marked 8^3 brick and clear its mark
__global__ void clear_kernel(float* __restrict__ fx, float* __restrict__ fy,
                             float* __restrict__ fz, uint8_t* __restrict__ bricks, int3 nb,
                             int nx, int ny, int nz) {
  const int lane = threadIdx.x & 31;
  const long nbt = (long)nb.x * nb.y * nb.z;
  const long wid = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long nw = ((long)gridDim.x * blockDim.x) >> 5;
  for (long bidx = wid; bidx < nbt; bidx += nw) {
    if (bricks[bidx] == 0) continue;
    const int bx = (int)(bidx % nb.x);
    const int by = (int)((bidx / nb.x) % nb.y);
    const int bz = (int)(bidx / ((long)nb.x * nb.y));
    // 512 cells per brick, 16 per lane: each warp store covers four whole
    // 8-float rows (four 32-byte sectors)
    for (int k = 0; k < 16; ++k) {
      const int idx = lane + 32 * k;
      const int xx = bx * 8 + (idx & 7), y = by * 8 + ((idx >> 3) & 7), z = bz * 8 + (idx >> 6);
      if (xx < nx && y < ny && z < nz) {
        const long o = ((long)z * ny + y) * nx + xx;
        fx[o] = 0.f;
        fy[o] = 0.f;
        fz[o] = 0.f;
      }
    }
    __syncwarp();
    if (lane == 0) bricks[bidx] = 0;
  }
}

template <bool M, bool I, bool P, bool S>
cudaError_t launch_t(ibm_ctx* c, const float* x, const float* v, const float* u, const float* vv,
                     const float* w, float* U, float* Fm, const float* Fm_in, float* Fext,
                     float* fx, float* fy, float* fz, uint8_t* bricks, int3 nb) {
  if (c->n_chunks == 0) return cudaSuccess;
  marker_kernel<M, I, P, S><<<c->n_chunks, kChunk, 0, c->stream>>>(
      c->d, c->grid, c->sc, (int32_t)c->V, (int32_t)c->F, x, v, u, vv, w, U, Fm, Fm_in, Fext,
      fx, fy, fz, bricks, nb);
  return cudaGetLastError();
}

}  // namespace

static int3 brick_dims(const ibm_ctx* c) {
  return make_int3((c->grid.n[0] + 7) / 8, (c->grid.n[1] + 7) / 8, (c->grid.n[2] + 7) / 8);
}

cudaError_t launch_mls(ibm_ctx* c, const float* x, const float* v, const float* u,
                       const float* vv, const float* w, float* U, float* Fm, const float* Fm_in,
                       float* Fext, float* fx, float* fy, float* fz, bool measure, bool interp,
                       bool probe, bool spread, bool record_cells) {
  const int3 nb = brick_dims(c);
  uint8_t* br = record_cells ? c->d_bricks : nullptr;
  if (measure && interp && probe && spread)
    return launch_t<true, true, true, true>(c, x, v, u, vv, w, U, Fm, Fm_in, Fext, fx, fy, fz, br, nb);
  if (measure && !interp && !probe && !spread)
    return launch_t<true, false, false, false>(c, x, v, u, vv, w, U, Fm, Fm_in, Fext, fx, fy, fz, br, nb);
  if (!measure && interp && probe && !spread)
    return launch_t<false, true, true, false>(c, x, v, u, vv, w, U, Fm, Fm_in, Fext, fx, fy, fz, br, nb);
  if (!measure && interp && !probe && !spread)
    return launch_t<false, true, false, false>(c, x, v, u, vv, w, U, Fm, Fm_in, Fext, fx, fy, fz, br, nb);
  if (!measure && !interp && probe && !spread)
    return launch_t<false, false, true, false>(c, x, v, u, vv, w, U, Fm, Fm_in, Fext, fx, fy, fz, br, nb);
  if (!measure && !interp && !probe && spread)
    return launch_t<false, false, false, true>(c, x, v, u, vv, w, U, Fm, Fm_in, Fext, fx, fy, fz, br, nb);
  return cudaErrorInvalidValue;
}

cudaError_t launch_clear(ibm_ctx* c, float* fx, float* fy, float* fz) {
  const int3 nb = brick_dims(c);
  clear_kernel<<<4 * 152, 256, 0, c->stream>>>(fx, fy, fz, c->d_bricks, nb, c->grid.n[0],
                                               c->grid.n[1], c->grid.n[2]);
  return cudaGetLastError();
}

}  // namespace ibm
