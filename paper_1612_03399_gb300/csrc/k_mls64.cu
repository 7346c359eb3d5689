// MLS interpolation with the general moment solve in float64 (Sec. 2.2,
// Eqs. mls..mls_Q): the option that keeps the whole interpolation, and the
// face geometry feeding it, in float64 on the GPU, beside the float32 closed
// form of the marker kernel.  It exists to measure what the float32 closed
// form costs in accuracy and saves in time.
//
// Per face (a thread each), per velocity component, at the centroid and at
// the probe end(s), with the 27 nodes of the component's nearest-node
// support (the same support as the marker kernel):
//   p_k = (1, s_k) with s_k the node offset from the support centre (cells),
//   W_k = exp(-kappa |s_k - t|^2) (the factorised Gaussian weight),
//   A = sum_k W_k p_k p_k^T, B_k = W_k p_k, p(t) = (1, t),
//   phi_k = p(t)^T A^-1 B_k,
// A factorised by LU with partial pivoting.  With r = A^-1 p(t) (A is
// symmetric) phi_k = W_k r . p_k, and the full derivative along e is
//   dphi_k/dt_e = W_k (q_e - m_e) . p_k + dW_k/dt_e r . p_k,
//   q_e = A^-1 dp/dt_e, m_e = A^-1 (dA/dt_e) r, dW_k/dt_e = 2 kappa (s_k,e - t_e) W_k,
// so one factorisation and seven 4x4 solves serve value and gradient.
// The probe traction is mu A (grad u + grad u^T) n (two-sided on open
// sheets), without pressure.  Velocities are read from global memory.
#include <cuda_runtime.h>
#include <math.h>

#include "ibm_internal.cuh"

namespace ibm {
namespace {

__device__ __forceinline__ int wrap64(int i, int n) {
  if (i >= 0 && i < n) return i;
  if (i < 0 && i >= -n) return i + n;
  if (i >= n && i < 2 * n) return i - n;
  i %= n;
  return i < 0 ? i + n : i;
}

// LU with partial pivoting of a 4x4 matrix (in place), permutation in piv
__device__ __forceinline__ void lu4(double (&a)[4][4], int (&piv)[4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i) piv[i] = i;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    int p = c;
    double best = fabs(a[c][c]);
#pragma unroll
    for (int r = c + 1; r < 4; ++r)
      if (fabs(a[r][c]) > best) {
        best = fabs(a[r][c]);
        p = r;
      }
    if (p != c) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const double t = a[c][j];
        a[c][j] = a[p][j];
        a[p][j] = t;
      }
      const int t = piv[c];
      piv[c] = piv[p];
      piv[p] = t;
    }
#pragma unroll
    for (int r = c + 1; r < 4; ++r) {
      const double f = a[r][c] / a[c][c];
      a[r][c] = f;
#pragma unroll
      for (int j = c + 1; j < 4; ++j) a[r][j] -= f * a[c][j];
    }
  }
}

__device__ __forceinline__ void lu_solve4(const double (&lu)[4][4], const int (&piv)[4],
                                          const double (&b)[4], double (&x)[4]) {
  double y[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    double s = b[piv[i]];
#pragma unroll
    for (int j = 0; j < i; ++j) s -= lu[i][j] * y[j];
    y[i] = s;
  }
#pragma unroll
  for (int i = 3; i >= 0; --i) {
    double s = y[i];
#pragma unroll
    for (int j = i + 1; j < 4; ++j) s -= lu[i][j] * x[j];
    x[i] = s / lu[i][i];
  }
}

// value (and, with grad, the gradient in cells) of the MLS interpolant of
// field f (component comp's lattice; comp 3: cell centres) at point t (cells,
// relative to the body's cell G)
template <bool GRAD>
__device__ void mls64(const float* __restrict__ f, const Grid& g, const double (&t)[3], int comp,
                      const int (&G)[3], double kappa, double& val, double (&gr)[3]) {
  int ic[3];
  double tl[3];   // point relative to the support centre (cells)
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double u = t[d] - (d == comp ? 0.0 : 0.5);
    const double c = floor(u + 0.5);
    tl[d] = u - c;
    ic[d] = G[d] + (int)c;
  }
  double A[4][4] = {};
  double dA[3][4][4] = {};
#pragma unroll 1
  for (int k = 0; k < 27; ++k) {
    const double s[3] = {(double)(k % 3 - 1), (double)((k / 3) % 3 - 1), (double)(k / 9 - 1)};
    const double d0 = s[0] - tl[0], d1 = s[1] - tl[1], d2 = s[2] - tl[2];
    const double W = exp(-kappa * (d0 * d0 + d1 * d1 + d2 * d2));
    const double p[4] = {1.0, s[0], s[1], s[2]};
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) A[i][j] += W * p[i] * p[j];
    if (GRAD) {
      const double dW[3] = {2.0 * kappa * d0 * W, 2.0 * kappa * d1 * W, 2.0 * kappa * d2 * W};
#pragma unroll
      for (int e = 0; e < 3; ++e)
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) dA[e][i][j] += dW[e] * p[i] * p[j];
    }
  }
  int piv[4];
  double lu[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) lu[i][j] = A[i][j];
  lu4(lu, piv);
  const double pt[4] = {1.0, tl[0], tl[1], tl[2]};
  double r[4];
  lu_solve4(lu, piv, pt, r);
  double qm[3][4];
  if (GRAD) {
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      double rhs[4] = {0.0, 0.0, 0.0, 0.0};
      rhs[e + 1] = 1.0;
      double q[4], m[4], dAr[4];
      lu_solve4(lu, piv, rhs, q);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        dAr[i] = 0.0;
#pragma unroll
        for (int j = 0; j < 4; ++j) dAr[i] += dA[e][i][j] * r[j];
      }
      lu_solve4(lu, piv, dAr, m);
#pragma unroll
      for (int i = 0; i < 4; ++i) qm[e][i] = q[i] - m[i];
    }
  }
  double v = 0.0, g0 = 0.0, g1 = 0.0, g2 = 0.0;
#pragma unroll 1
  for (int k = 0; k < 27; ++k) {
    const int sx = k % 3 - 1, sy = (k / 3) % 3 - 1, sz = k / 9 - 1;
    const double s[3] = {(double)sx, (double)sy, (double)sz};
    const double d0 = s[0] - tl[0], d1 = s[1] - tl[1], d2 = s[2] - tl[2];
    const double W = exp(-kappa * (d0 * d0 + d1 * d1 + d2 * d2));
    const double p[4] = {1.0, s[0], s[1], s[2]};
    const double rp = r[0] * p[0] + r[1] * p[1] + r[2] * p[2] + r[3] * p[3];
    const size_t idx = ((size_t)wrap64(ic[2] + sz, g.n[2]) * g.n[1] + wrap64(ic[1] + sy, g.n[1])) *
                           g.n[0] + wrap64(ic[0] + sx, g.n[0]);
    const double q = (double)__ldg(f + idx);
    v += W * rp * q;
    if (GRAD) {
      const double dW[3] = {2.0 * kappa * d0 * W, 2.0 * kappa * d1 * W, 2.0 * kappa * d2 * W};
      double dphi[3];
#pragma unroll
      for (int e = 0; e < 3; ++e)
        dphi[e] = W * (qm[e][0] * p[0] + qm[e][1] * p[1] + qm[e][2] * p[2] + qm[e][3] * p[3]) +
                  dW[e] * rp;
      g0 += dphi[0] * q;
      g1 += dphi[1] * q;
      g2 += dphi[2] * q;
    }
  }
  val = v;
  gr[0] = g0;
  gr[1] = g1;
  gr[2] = g2;
}

struct Spacing64 {
  double h[3];
};

__global__ void __launch_bounds__(kMT) interp64_kernel(
    DeviceTables T, Grid g, Spacing64 hs, double dt, double mu, double kappa, double probe_h,
    int32_t V, int32_t F,
    const float* __restrict__ x, const float* __restrict__ v, const float* __restrict__ u,
    const float* __restrict__ vv, const float* __restrict__ w, float* __restrict__ U,
    float* __restrict__ Fm, float* __restrict__ Fext) {
  const int4 ch = T.chunks[blockIdx.x];
  if ((int)threadIdx.x >= ch.z) return;
  const BodyDev B = T.body[ch.x];
  const TopoDev topo = T.topo[B.topo];
  const int4 mt = __ldg(T.mtri + topo.mface_off + ch.y + threadIdx.x);
  const int gf = B.f_off + mt.w;
  const int ia = B.v_off + mt.x, ib = B.v_off + mt.y, ic = B.v_off + mt.z;
  double xa[3], xb[3], xc[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    xa[d] = (double)__ldg(x + d * V + ia);
    xb[d] = (double)__ldg(x + d * V + ib);
    xc[d] = (double)__ldg(x + d * V + ic);
  }
  const double e1[3] = {xb[0] - xa[0], xb[1] - xa[1], xb[2] - xa[2]};
  const double e2[3] = {xc[0] - xa[0], xc[1] - xa[1], xc[2] - xa[2]};
  const double N[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                       e1[0] * e2[1] - e1[1] * e2[0]};
  const double nn = sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
  if (!(nn > 0.0)) {
    atomicOr(T.err, ERR_NONFINITE);
    return;
  }
  const double area = 0.5 * nn;
  double n[3], tc[3], tp[3], tm[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    n[d] = N[d] / nn;
    const double c = (xa[d] + xb[d] + xc[d]) / 3.0;
    tc[d] = c / hs.h[d] + B.fracd[d];
    tp[d] = (c + probe_h * n[d]) / hs.h[d] + B.fracd[d];
    tm[d] = (c - probe_h * n[d]) / hs.h[d] + B.fracd[d];
    if (!(fabs(tc[d]) < 4.0e6 && fabs(tp[d]) < 4.0e6)) {
      atomicOr(T.err, ERR_NONFINITE);
      return;
    }
  }
  const float* fld[3] = {u, vv, w};
  double G[3][3];
#pragma unroll 1
  for (int i = 0; i < 3; ++i) {
    double val, gr[3];
    if (U || Fm) {
      mls64<false>(fld[i], g, tc, i, B.G, kappa, val, gr);
      if (U) U[i * F + gf] = (float)val;
      if (Fm) {
        const double vb = ((double)__ldg(v + i * V + ia) + (double)__ldg(v + i * V + ib) +
                           (double)__ldg(v + i * V + ic)) / 3.0;
        Fm[i * F + gf] = (float)((vb - val) / dt);
      }
    }
    if (Fext) {
      mls64<true>(fld[i], g, tp, i, B.G, kappa, val, gr);
#pragma unroll
      for (int j = 0; j < 3; ++j) G[i][j] = gr[j] / hs.h[j];
      if (!B.closed) {
        mls64<true>(fld[i], g, tm, i, B.G, kappa, val, gr);
#pragma unroll
        for (int j = 0; j < 3; ++j) G[i][j] -= gr[j] / hs.h[j];
      }
    }
  }
  if (Fext) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      double t = 0.0;
#pragma unroll
      for (int j = 0; j < 3; ++j) t += (G[i][j] + G[j][i]) * n[j];
      Fext[i * F + gf] = (float)(mu * area * t);
    }
  }
}

}  // namespace

cudaError_t launch_interp64(ibm_ctx* c, const float* x, const float* v, const float* u,
                            const float* vv, const float* w, float* U, float* Fm, float* Fext) {
  if (c->n_chunks == 0) return cudaSuccess;
  const double alpha = c->prm.alpha > 0 ? c->prm.alpha : 0.3;
  const double kappa = 1.0 / ((1.5 * alpha) * (1.5 * alpha));
  double probe_h = c->prm.probe_h;
  if (!(probe_h > 0)) {
    probe_h = 0.0;
    for (int d = 0; d < 3; ++d) probe_h += c->gdesc.L[d] / c->gdesc.n[d];
    probe_h /= 3.0;
  }
  Spacing64 hs;
  for (int d = 0; d < 3; ++d) hs.h[d] = c->gdesc.L[d] / c->gdesc.n[d];
  interp64_kernel<<<c->n_chunks, kMT, 0, c->stream>>>(c->d, c->grid, hs, c->prm.dt, c->prm.mu,
                                                      kappa, probe_h,
                                                      (int32_t)c->V, (int32_t)c->F, x, v, u, vv,
                                                      w, U, Fm, Fext);
  return cudaGetLastError();
}

}  // namespace ibm
