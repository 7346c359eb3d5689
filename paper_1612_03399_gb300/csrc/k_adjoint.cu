// Adjoint of one step (a vector-Jacobian product): given the cotangents
// (gx', gv') of the new positions and velocities, the cotangents (gx, gv) of
// the old ones and of the per-body elastic constants.
//
// The step (Sec. 2.3, Sec. 5 step 4) is v' = v + dt F(x)/m, x' = x + dt v'
// (symplectic) or x' = x + dt v (forward Euler), F = F_int + F_ext^v; clamped
// nodes keep x and get v' = 0.  So gv = gv' + dt gx', the force cotangent is
// gF = dt (gv' + dt gx')/m (symplectic) or dt gv'/m (forward Euler), zero on
// clamped nodes, and gx = gx' + (dF_int/dx)^T gF + (dF_ext^v/dx)^T gF.
//
// With cotangents g of the spread force fields (Eq. mls_cl), the spread's
// dependence on x (centroid and area of every face) and on v (the face's
// centroid velocity in the marker force) is added as well.
//
// ext_adjoint_kernel (per face): the traction F_ext = mu A (G + G^T) n at the
// probe end p = c + h n (two probes on open sheets) depends on x through A,
// n, c and the MLS velocity gradient G(p); its reverse sweep needs the
// second derivatives of the MLS interpolant at p.  It also sums, per body,
// grad A . gF and grad V . gF (fixed order), which the global area and
// volume terms need.
//
// force_adjoint_kernel (per force patch): the element forces evaluated with
// dual numbers whose tangents are gF give (dF_int/dx) gF (= its transpose:
// F_int is minus an energy gradient, so its Jacobian is symmetric); the
// constants' cotangents are gF . dF/dk, summed per body in a fixed order.
#include <cuda_runtime.h>

#include "bulk_copy.cuh"
#include "force_elems.cuh"
#include "ibm_internal.cuh"

namespace ibm {
namespace {

__device__ __forceinline__ int wrap(int i, int n) {
  if (i >= 0 && i < n) return i;
  if (i < 0 && i >= -n) return i + n;
  if (i >= n && i < 2 * n) return i - n;
  i %= n;
  return i < 0 ? i + n : i;
}

// per-direction MLS factors a, b = a beta and their first and second
// derivatives with respect to the point's coordinate in cells (closed form
// of the factorised weight; see the marker kernel)
struct DirW2 {
  float a[3][3], b[3][3];   // [order][node]
};
__device__ __forceinline__ void dir_weights_d2(float tp, float kappa, DirW2& o) {
  float d[3] = {-1.f - tp, -tp, 1.f - tp};
  float w[3], w1[3], w2[3];
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    w[s] = __expf(-kappa * d[s] * d[s]);
    w1[s] = 2.f * kappa * d[s] * w[s];
    w2[s] = 2.f * kappa * w[s] * (2.f * kappa * d[s] * d[s] - 1.f);
  }
  const float invS = 1.f / (w[0] + w[1] + w[2]);
  const float S1 = w1[0] + w1[1] + w1[2], S2 = w2[0] + w2[1] + w2[2];
  float a[3], a1[3], a2[3];
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    a[s] = w[s] * invS;
    a1[s] = (w1[s] - a[s] * S1) * invS;
  }
#pragma unroll
  for (int s = 0; s < 3; ++s) a2[s] = (w2[s] - 2.f * a1[s] * S1 - a[s] * S2) * invS;
  float mu = 0.f, mu1 = -1.f, mu2 = 0.f;
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    mu += a[s] * d[s];
    mu1 += a1[s] * d[s];
    mu2 += a2[s] * d[s] - a1[s];
  }
  const float e1 = -1.f - mu1, e2 = -mu2;   // derivatives of e_s = d_s - mu (same for all s)
  float Q = 0.f, Q1 = 0.f, Q2 = 0.f;
  float e[3];
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    e[s] = d[s] - mu;
    Q += a[s] * e[s] * e[s];
    Q1 += a1[s] * e[s] * e[s] + 2.f * a[s] * e[s] * e1;
    Q2 += a2[s] * e[s] * e[s] + 4.f * a1[s] * e[s] * e1 + 2.f * a[s] * e1 * e1 + 2.f * a[s] * e[s] * e2;
  }
  const float iQ = 1.f / Q;
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const float P = mu * e[s], P1 = mu1 * e[s] + mu * e1, P2 = mu2 * e[s] + 2.f * mu1 * e1 + mu * e2;
    const float beta = P * iQ;
    const float beta1 = P1 * iQ - P * Q1 * iQ * iQ;
    const float beta2 = P2 * iQ - 2.f * P1 * Q1 * iQ * iQ - P * Q2 * iQ * iQ +
                        2.f * P * Q1 * Q1 * iQ * iQ * iQ;
    o.a[0][s] = a[s];
    o.a[1][s] = a1[s];
    o.a[2][s] = a2[s];
    o.b[0][s] = a[s] * beta;
    o.b[1][s] = a1[s] * beta + a[s] * beta1;
    o.b[2][s] = a2[s] * beta + 2.f * a1[s] * beta1 + a[s] * beta2;
  }
}

// gradient (cells) and Hessian (cells; xx, yy, zz, xy, xz, yz) of the MLS
// interpolant of one velocity component at a point
__device__ void mls_grad_hess(const float* __restrict__ f, const Grid& g, const float (&tau)[3],
                              int comp, const int (&G)[3], float kappa, float (&gr)[3],
                              float (&hs)[6]) {
  int c[3];
  float tp[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float uu = tau[d] - (d == comp ? 0.f : 0.5f);
    const float cc = floorf(uu + 0.5f);
    tp[d] = uu - cc;
    c[d] = G[d] + (int)cc;
  }
  DirW2 X, Y, Z;
  dir_weights_d2(tp[0], kappa, X);
  dir_weights_d2(tp[1], kappa, Y);
  dir_weights_d2(tp[2], kappa, Z);
  int ix[3], iy[3], iz[3];
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    ix[s] = wrap(c[0] - 1 + s, g.n[0]);
    iy[s] = wrap(c[1] - 1 + s, g.n[1]);
    iz[s] = wrap(c[2] - 1 + s, g.n[2]);
  }
  // nine derivative patterns (x, y, z orders): 100 010 001 200 020 002 110
  // 101 011.  Separable contraction: per row the (a, b) sums of the three x
  // orders as packed pairs; per z-plane, for the six (x, y) order pairs the
  // patterns use, P = sum_y a_y (xa, xb) and P3 = sum_y b_y xa; then per
  // pattern acc += a_z (P.x - P.y - P3) - b_z P.x
  constexpr int GX[6] = {1, 0, 0, 2, 0, 1}, GY[6] = {0, 1, 0, 0, 2, 1};
  float acc[9];
#pragma unroll
  for (int p = 0; p < 9; ++p) acc[p] = 0.f;
#pragma unroll
  for (int sz = 0; sz < 3; ++sz) {
    float2 P[6];
    float P3[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      P[q] = make_float2(0.f, 0.f);
      P3[q] = 0.f;
    }
#pragma unroll
    for (int sy = 0; sy < 3; ++sy) {
      const float* r = f + ((size_t)iz[sz] * g.n[1] + iy[sy]) * g.n[0];
      const float u0 = __ldg(r + ix[0]), u1 = __ldg(r + ix[1]), u2 = __ldg(r + ix[2]);
      float2 xo[3];
#pragma unroll
      for (int o = 0; o < 3; ++o) {
        xo[o] = __fmul2_rn(make_float2(X.a[o][0], X.b[o][0]), make_float2(u0, u0));
        xo[o] = __ffma2_rn(make_float2(X.a[o][1], X.b[o][1]), make_float2(u1, u1), xo[o]);
        xo[o] = __ffma2_rn(make_float2(X.a[o][2], X.b[o][2]), make_float2(u2, u2), xo[o]);
      }
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        const float ay = Y.a[GY[q]][sy];
        P[q] = __ffma2_rn(make_float2(ay, ay), xo[GX[q]], P[q]);
        P3[q] = fmaf(Y.b[GY[q]][sy], xo[GX[q]].x, P3[q]);
      }
    }
    // pattern p: (x, y) pair and z order
    constexpr int PQ[9] = {0, 1, 2, 3, 4, 2, 5, 0, 1}, PZ[9] = {0, 0, 1, 0, 0, 2, 0, 1, 1};
#pragma unroll
    for (int p = 0; p < 9; ++p) {
      const int q = PQ[p];
      acc[p] = fmaf(Z.a[PZ[p]][sz], P[q].x - P[q].y - P3[q], fmaf(-Z.b[PZ[p]][sz], P[q].x, acc[p]));
    }
  }
  gr[0] = acc[0];
  gr[1] = acc[1];
  gr[2] = acc[2];
#pragma unroll
  for (int k = 0; k < 6; ++k) hs[k] = acc[3 + k];
}

// value and gradient (cells) of the MLS interpolant of one field at a point
// (comp 0-2: velocity lattices, 3: cell centres)
__device__ void mls_val_grad(const float* __restrict__ f, const Grid& g, const float (&tau)[3],
                             int comp, const int (&G)[3], float kappa, float& val,
                             float (&gr)[3]) {
  int c[3];
  float tp[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float uu = tau[d] - (d == comp ? 0.f : 0.5f);
    const float cc = floorf(uu + 0.5f);
    tp[d] = uu - cc;
    c[d] = G[d] + (int)cc;
  }
  DirW2 X, Y, Z;
  dir_weights_d2(tp[0], kappa, X);
  dir_weights_d2(tp[1], kappa, Y);
  dir_weights_d2(tp[2], kappa, Z);
  int ix[3], iy[3], iz[3];
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    ix[s] = wrap(c[0] - 1 + s, g.n[0]);
    iy[s] = wrap(c[1] - 1 + s, g.n[1]);
    iz[s] = wrap(c[2] - 1 + s, g.n[2]);
  }
  // value and the three first derivatives (patterns 000 100 010 001), with
  // the separable contraction of mls_grad_hess: (x, y) order pairs 00, 10, 01
  constexpr int GX[3] = {0, 1, 0}, GY[3] = {0, 0, 1};
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int sz = 0; sz < 3; ++sz) {
    float2 P[3];
    float P3[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      P[q] = make_float2(0.f, 0.f);
      P3[q] = 0.f;
    }
#pragma unroll
    for (int sy = 0; sy < 3; ++sy) {
      const float* r = f + ((size_t)iz[sz] * g.n[1] + iy[sy]) * g.n[0];
      const float u0 = __ldg(r + ix[0]), u1 = __ldg(r + ix[1]), u2 = __ldg(r + ix[2]);
      float2 xo[2];
#pragma unroll
      for (int o = 0; o < 2; ++o) {
        xo[o] = __fmul2_rn(make_float2(X.a[o][0], X.b[o][0]), make_float2(u0, u0));
        xo[o] = __ffma2_rn(make_float2(X.a[o][1], X.b[o][1]), make_float2(u1, u1), xo[o]);
        xo[o] = __ffma2_rn(make_float2(X.a[o][2], X.b[o][2]), make_float2(u2, u2), xo[o]);
      }
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const float ay = Y.a[GY[q]][sy];
        P[q] = __ffma2_rn(make_float2(ay, ay), xo[GX[q]], P[q]);
        P3[q] = fmaf(Y.b[GY[q]][sy], xo[GX[q]].x, P3[q]);
      }
    }
    constexpr int PQ[4] = {0, 1, 2, 0}, PZ[4] = {0, 0, 0, 1};
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int q = PQ[p];
      acc[p] = fmaf(Z.a[PZ[p]][sz], P[q].x - P[q].y - P3[q], fmaf(-Z.b[PZ[p]][sz], P[q].x, acc[p]));
    }
  }
  val = acc[0];
  gr[0] = acc[1];
  gr[1] = acc[2];
  gr[2] = acc[3];
}

__device__ __forceinline__ float hess_at(const float (&hs)[6], int j, int k) {
  if (j == k) return hs[j];
  const int m = j + k;   // (0,1) -> 1, (0,2) -> 2, (1,2) -> 3
  return hs[2 + m];
}

// force cotangent of vertex gv: dt (gv' + dt gx')/m (symplectic) or dt gv'/m
__device__ __forceinline__ void force_cot(const DeviceTables& T, const StepConsts& sc, int V, int gv,
                                          float inv_mass, const float* __restrict__ gxn,
                                          const float* __restrict__ gvn, float (&o)[3]) {
  if (T.clamp[gv]) {
    o[0] = o[1] = o[2] = 0.f;
    return;
  }
  const float s = sc.dt * inv_mass;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float gvv = __ldg(gvn + d * V + gv);
    o[d] = sc.forward_euler ? s * gvv : s * (gvv + sc.dt * __ldg(gxn + d * V + gv));
  }
}

__device__ __forceinline__ void cross3(const float (&a)[3], const float (&b)[3], float (&o)[3]) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

__global__ void __launch_bounds__(kMT, 2) ext_adjoint_kernel(
    DeviceTables T, Grid g, StepConsts sc, int32_t V, int32_t F, const float* __restrict__ x,
    const float* __restrict__ vel, const float* __restrict__ u, const float* __restrict__ vv,
    const float* __restrict__ w, const float* __restrict__ pr, const float* __restrict__ accel,
    const float* __restrict__ gxn, const float* __restrict__ gvn, const float* __restrict__ gfx,
    const float* __restrict__ gfy, const float* __restrict__ gfz, float* __restrict__ gve) {
  __shared__ double s_red[2][kMT / 32];
  __shared__ int s_last;
  const int4 ch = T.chunks[blockIdx.x];
  const BodyDev B = T.body[ch.x];
  const TopoDev topo = T.topo[B.topo];
  double dA = 0.0, dV = 0.0;
  if ((int)threadIdx.x < ch.z) {
    const int lf = __ldg(T.mface + topo.mface_off + ch.y + threadIdx.x);
    const int gf = B.f_off + lf;
    const int* tr = T.tri + topo.tri_off + 3 * lf;
    const int id[3] = {B.v_off + __ldg(tr), B.v_off + __ldg(tr + 1), B.v_off + __ldg(tr + 2)};
    float p[3][3], ga[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
#pragma unroll
      for (int d = 0; d < 3; ++d) p[k][d] = __ldg(x + d * V + id[k]);
      force_cot(T, sc, V, id[k], B.inv_mass, gxn, gvn, ga[k]);
    }
    float e1[3], e2[3], N[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      e1[d] = p[1][d] - p[0][d];
      e2[d] = p[2][d] - p[0][d];
    }
    cross3(e1, e2, N);
    const float nn = sqrtf(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
    const float area = 0.5f * nn, inv = 1.f / nn;
    const float n[3] = {N[0] * inv, N[1] * inv, N[2] * inv};
    // per-body sums grad A . gF and grad V . gF
    {
      float gVv[3], t[3];
      const float cb[3] = {p[2][0] - p[1][0], p[2][1] - p[1][1], p[2][2] - p[1][2]};
      const float ac[3] = {p[0][0] - p[2][0], p[0][1] - p[2][1], p[0][2] - p[2][2]};
      const float ba[3] = {p[1][0] - p[0][0], p[1][1] - p[0][1], p[1][2] - p[0][2]};
      float sA = 0.f, sV = 0.f;
      cross3(n, cb, t);
      sA += 0.5f * (t[0] * ga[0][0] + t[1] * ga[0][1] + t[2] * ga[0][2]);
      cross3(n, ac, t);
      sA += 0.5f * (t[0] * ga[1][0] + t[1] * ga[1][1] + t[2] * ga[1][2]);
      cross3(n, ba, t);
      sA += 0.5f * (t[0] * ga[2][0] + t[1] * ga[2][1] + t[2] * ga[2][2]);
      if (B.closed) {
        cross3(p[1], p[2], gVv);
        sV += (gVv[0] * ga[0][0] + gVv[1] * ga[0][1] + gVv[2] * ga[0][2]) * (1.f / 6.f);
        cross3(p[2], p[0], gVv);
        sV += (gVv[0] * ga[1][0] + gVv[1] * ga[1][1] + gVv[2] * ga[1][2]) * (1.f / 6.f);
        cross3(p[0], p[1], gVv);
        sV += (gVv[0] * ga[2][0] + gVv[1] * ga[2][1] + gVv[2] * ga[2][2]) * (1.f / 6.f);
      }
      dA = sA;
      dV = sV;
    }
    // traction cotangent: F_ext^v = sum over faces F_ext/3
    float gF[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) gF[d] = (ga[0][d] + ga[1][d] + ga[2][d]) * (1.f / 3.f);
    const float third = 1.f / 3.f;
    float c[3], tpp[3], tpm[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      c[d] = (p[0][d] + p[1][d] + p[2][d]) * third;
      tpp[d] = fmaf(c[d] + sc.probe_h * n[d], g.invh[d], B.frac[d]);
      tpm[d] = fmaf(c[d] - sc.probe_h * n[d], g.invh[d], B.frac[d]);
    }
    const bool two = !B.closed;
    const float* fld[3] = {u, vv, w};
    // one gradient-and-Hessian evaluation per component and probe end: the
    // gradient forms G, the Hessian the position cotangent of the probe ends,
    // gp_k = sum_ij gG_ij H_ijk with gG_ij = mu A (gF_i n_j + gF_j n_i), which
    // does not depend on G
    float G[3][3];
    float gpp[3] = {0.f, 0.f, 0.f}, gpm[3] = {0.f, 0.f, 0.f};
    const float s = sc.mu * area;
#pragma unroll 1
    for (int i = 0; i < 3; ++i) {
      float gr[3], hs[6];
      mls_grad_hess(fld[i], g, tpp, i, B.G, sc.kappa, gr, hs);
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        G[i][j] = gr[j] * g.invh[j];
        const float gG = s * (gF[i] * n[j] + gF[j] * n[i]);
#pragma unroll
        for (int k = 0; k < 3; ++k) gpp[k] += gG * hess_at(hs, j, k) * g.invh[j] * g.invh[k];
      }
      if (two) {
        mls_grad_hess(fld[i], g, tpm, i, B.G, sc.kappa, gr, hs);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          G[i][j] -= gr[j] * g.invh[j];
          const float gG = s * (gF[i] * n[j] + gF[j] * n[i]);
#pragma unroll
          for (int k = 0; k < 3; ++k) gpm[k] -= gG * hess_at(hs, j, k) * g.invh[j] * g.invh[k];
        }
      }
    }
    // F = mu A (G + G^T) n
    float Tn[3], TgF[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      Tn[i] = 0.f;
      TgF[i] = 0.f;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const float Tij = G[i][j] + G[j][i];
        Tn[i] += Tij * n[j];
        TgF[i] += Tij * gF[j];
      }
    }
    float gArea = sc.mu * (gF[0] * Tn[0] + gF[1] * Tn[1] + gF[2] * Tn[2]);
    float gn[3] = {sc.mu * area * TgF[0], sc.mu * area * TgF[1], sc.mu * area * TgF[2]};
    // p+- = c +- h n
    float gc[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      gc[d] = gpp[d] + gpm[d];
      gn[d] += sc.probe_h * (gpp[d] - gpm[d]);
    }
    if (pr) {
      // pressure load -A P n with P = p*(c + h n) [- p*(c - h n)] + k h a.n,
      // k = 1 (closed) or 2 (open; each side with its own normal); the
      // marker acceleration a is an input and is held fixed
      float am[3] = {0.f, 0.f, 0.f};
      if (accel) {
#pragma unroll
        for (int d = 0; d < 3; ++d)
          am[d] = (__ldg(accel + d * V + id[0]) + __ldg(accel + d * V + id[1]) +
                   __ldg(accel + d * V + id[2])) * third;
      }
      float P, gpr[3], dPdc[3], dPdn[3];
      mls_val_grad(pr, g, tpp, 3, B.G, sc.kappa, P, gpr);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        dPdc[d] = gpr[d] * g.invh[d];
        dPdn[d] = sc.probe_h * dPdc[d];
      }
      if (two) {
        float Pm;
        mls_val_grad(pr, g, tpm, 3, B.G, sc.kappa, Pm, gpr);
        P -= Pm;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const float gd = gpr[d] * g.invh[d];
          dPdc[d] -= gd;
          dPdn[d] += sc.probe_h * gd;
        }
      }
      const float kh = (two ? 2.f : 1.f) * sc.probe_h;
      P += kh * (am[0] * n[0] + am[1] * n[1] + am[2] * n[2]);
      const float gFn = gF[0] * n[0] + gF[1] * n[1] + gF[2] * n[2];
      gArea -= P * gFn;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        gn[d] -= area * (P * gF[d] + gFn * (dPdn[d] + kh * am[d]));
        gc[d] -= area * gFn * dPdc[d];
      }
    }
    if (gfx) {
      // the spread f_i^k = c_l phi_k(c) F_i with F_i = (V^b_i - U_i(c))/dt,
      // c_l = A cl_scale (Eq. mls_cl), against the field cotangents g_i: with
      // G_i = sum_k phi_k(c) g_i^k (spreading transposed is interpolation),
      // dL/dF_i = c_l G_i, so the vertex velocities get c_l G_i / (3 dt)
      // each, the centroid c_l (F_i grad G_i - G_i grad U_i / dt) and the
      // area cl_scale sum_i F_i G_i
      const float* gfs[3] = {gfx, gfy, gfz};
      float tcc[3], vb[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        tcc[d] = fmaf(c[d], g.invh[d], B.frac[d]);
        vb[d] = (__ldg(vel + d * V + id[0]) + __ldg(vel + d * V + id[1]) +
                 __ldg(vel + d * V + id[2])) * third;
      }
      const float cl = area * sc.cl_scale;
      float gAs = 0.f;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        float Uv, Ug[3], Gv, Gg[3];
        mls_val_grad(fld[i], g, tcc, i, B.G, sc.kappa, Uv, Ug);
        mls_val_grad(gfs[i], g, tcc, i, B.G, sc.kappa, Gv, Gg);
        const float Fi = (vb[i] - Uv) * sc.inv_dt;
        gAs += Fi * Gv;
#pragma unroll
        for (int d = 0; d < 3; ++d) gc[d] += cl * (Fi * Gg[d] - Gv * sc.inv_dt * Ug[d]) * g.invh[d];
        gve[i * (size_t)F + gf] = cl * Gv * sc.inv_dt * third;
      }
      gArea += sc.cl_scale * gAs;
    }
    // n = N/|N|, A = |N|/2
    const float gnn = gn[0] * n[0] + gn[1] * n[1] + gn[2] * n[2];
    float gN[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) gN[d] = (gn[d] - gnn * n[d]) * inv + 0.5f * gArea * n[d];
    // N = e1 x e2
    float ge1[3], ge2[3];
    cross3(e2, gN, ge1);
    cross3(gN, e1, ge2);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const float gcd = gc[d] * third;
      T.gxe[(0 * 3 + d) * (size_t)F + gf] = -ge1[d] - ge2[d] + gcd;
      T.gxe[(1 * 3 + d) * (size_t)F + gf] = ge1[d] + gcd;
      T.gxe[(2 * 3 + d) * (size_t)F + gf] = ge2[d] + gcd;
    }
  }
  // fixed-order per-body sums of grad A . gF and grad V . gF
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    dA += __shfl_down_sync(0xffffffffu, dA, o);
    dV += __shfl_down_sync(0xffffffffu, dV, o);
  }
  if ((threadIdx.x & 31) == 0) {
    s_red[0][threadIdx.x >> 5] = dA;
    s_red[1][threadIdx.x >> 5] = dV;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < kMT / 32; ++k) {
      a += s_red[0][k];
      b += s_red[1][k];
    }
    const int gc = B.chunk_off + ch.w;
    T.partial2[2 * gc] = a;
    T.partial2[2 * gc + 1] = b;
    __threadfence();
    s_last = (atomicAdd(T.counter2 + ch.x, 1) == B.n_chunk - 1);
  }
  __syncthreads();
  if (s_last && threadIdx.x == 0) {
    __threadfence();
    const volatile double* P = T.partial2;
    double a = 0.0, b = 0.0;
    for (int k = 0; k < B.n_chunk; ++k) {
      a += P[2 * (B.chunk_off + k)];
      b += P[2 * (B.chunk_off + k) + 1];
    }
    T.dmeas[2 * ch.x] = a;
    T.dmeas[2 * ch.x + 1] = b;
    T.counter2[ch.x] = 0;
  }
}

struct DSmem {
  float *px, *py, *pz, *tx, *ty, *tz, *cx, *cy, *cz;
  __device__ Vec<Dual> pos(int i) const {
    return {Dual(px[i], tx[i]), Dual(py[i], ty[i]), Dual(pz[i], tz[i])};
  }
  __device__ Vec<float> cot(int i) const { return {tx[i], ty[i], tz[i]}; }
  __device__ void put(int s, const Vec<Dual>& f) const {
    if (s == kNone) return;
    cx[s] = f.x.d;
    cy[s] = f.y.d;
    cz[s] = f.z.d;
  }
  __device__ void add(int s, const Vec<Dual>& f) const {
    if (s == kNone) return;
    cx[s] += f.x.d;
    cy[s] += f.y.d;
    cz[s] += f.z.d;
  }
};

__device__ __forceinline__ float dotv(const Vec<float>& a, const Vec<Dual>& b) {
  return a.x * b.x.v + a.y * b.y.v + a.z * b.z.v;
}

__global__ void __launch_bounds__(kForceThreads) force_adjoint_kernel(
    DeviceTables T, StepConsts sc, int32_t V, int32_t F, const float* __restrict__ x,
    const float* __restrict__ gxn, const float* __restrict__ gvn, float* __restrict__ gx,
    float* __restrict__ gvo, double* __restrict__ gparams, const float* __restrict__ gve) {
  extern __shared__ __align__(16) float sm[];
  __shared__ double s_red[3][kForceThreads / 32];
  __shared__ int s_last;
  __shared__ __align__(8) unsigned long long bar;
  const int2 wk = T.work[blockIdx.x];
  const BodyDev B = T.body[wk.x];
  const TopoDev topo = T.topo[B.topo];
  const PatchHdr P = T.patch[topo.patch_off + wk.y];
  const FPatch Q = T.fpatch[topo.patch_off + wk.y];
  // the forward kernel's blob (edge and face records, slot starts) with the
  // adjoint's tail (each own vertex's faces and corners), the rest data,
  // positions and tangents of the local vertices, contribution slots
  const int pe = pad4(P.n_edge), pf = pad4(P.n_face);
  const int rest_words = frest_words(P.n_edge, P.n_face, B.varied != 0);
  const uint4* rec = reinterpret_cast<const uint4*>(sm);
  const uint2* frec = reinterpret_cast<const uint2*>(sm + 4 * P.n_edge);
  const uint16_t* ptr = reinterpret_cast<const uint16_t*>(sm + 4 * P.n_edge + 2 * P.n_face);
  const uint16_t* vptr = reinterpret_cast<const uint16_t*>(sm + Q.blob_words);
  const uint32_t* vent = reinterpret_cast<const uint32_t*>(sm + Q.blob_words) + (P.n_own + 2) / 2;
  const float* rest = sm + Q.blob_words + Q.vf_words;
  DSmem S;
  S.px = sm + Q.blob_words + Q.vf_words + rest_words;
  S.py = S.px + pad4(P.n_loc);
  S.pz = S.py + pad4(P.n_loc);
  S.tx = S.pz + pad4(P.n_loc);
  S.ty = S.tx + pad4(P.n_loc);
  S.tz = S.ty + pad4(P.n_loc);
  S.cx = S.tz + pad4(P.n_loc);
  S.cy = S.cx + pad4(Q.n_slot);
  S.cz = S.cy + pad4(Q.n_slot);
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    const unsigned nb = 4u * (unsigned)(Q.blob_words + Q.vf_words), nr = 4u * (unsigned)rest_words;
    mbar_arrive_tx(&bar, nb + nr + (unsigned)sc.starve_tx);
    if (nb) bulk_load(sm, T.fblob + Q.blob_off, nb, &bar);
    if (nr) bulk_load(sm + Q.blob_words + Q.vf_words, T.frest + T.wrest[blockIdx.x], nr, &bar);
  }
  for (int i = threadIdx.x; i < P.n_loc; i += blockDim.x) {
    const int gvx = B.v_off + __ldg(T.loc_vert + P.loc_off + i);
    S.px[i] = __ldg(x + gvx);
    S.py[i] = __ldg(x + V + gvx);
    S.pz[i] = __ldg(x + 2 * V + gvx);
    float o[3];
    force_cot(T, sc, V, gvx, B.inv_mass, gxn, gvn, o);
    S.tx[i] = o[0];
    S.ty[i] = o[1];
    S.tz[i] = o[2];
  }
  // global-term coefficients and their derivatives along gF
  const float2 cf = T.coef[wk.x];
  const double dA = T.dmeas[2 * wk.x], dV = T.dmeas[2 * wk.x + 1];
  const Dual cA(cf.x, (float)(B.kA / B.A0 * dA));
  const Dual cV(cf.y, B.closed ? (float)(B.kv / B.V0 * dV) : 0.f);
  double gks = 0.0, gkb = 0.0, gka = 0.0;
  __syncthreads();   // positions and tangents staged, barrier initialised
  if (!__syncthreads_and(mbar_wait(&bar, kCopyWaitClocks))) {
    // the copies did not land: flag it, give them one more bounded wait
    // (they write this block's shared memory) and leave
    if (threadIdx.x == 0) {
      atomicOr(T.err, ERR_TIMEOUT);
      mbar_wait(&bar, kCopyWaitClocks);
    }
    __syncthreads();
    return;
  }
  for (int k = threadIdx.x; k < P.n_edge; k += blockDim.x) {
    const uint4 r = rec[k];
    const int la = r.x & 0xFFFF, lb = r.x >> 16, lc = r.y & 0xFFFF, ld = r.y >> 16;
    const bool hinge = ld != kNone;
    const Vec<Dual> pa = S.pos(la), pb = S.pos(lb);
    const Vec<Dual> pc = hinge ? S.pos(lc) : pa, pd = hinge ? S.pos(ld) : pb;
    const float c0 = hinge ? rest[pe + k] : 1.f, s0 = hinge ? rest[2 * pe + k] : 0.f;
    Vec<Dual> fa, fb, fc, fd, us[2], ub[4];
    float es, eb;
    // per-edge multipliers m: the forces use m k, the constants' cotangents
    // scale the per-unit-k forces by m
    const float ms = B.varied ? rest[3 * pe + pf + k] : 1.f;
    const float mb = B.varied ? rest[4 * pe + pf + k] : 1.f;
    edge_forces(pa, pb, pc, pd, hinge, rest[k], c0, s0, B.ks * ms, B.kb * mb, fa, fb, fc, fd, us,
                ub, es, eb);
    S.put(r.z & 0xFFFF, fa);
    S.put(r.z >> 16, fb);
    S.put(r.w & 0xFFFF, fc);
    S.put(r.w >> 16, fd);
    if ((r.z & 0xFFFF) != kNone) {   // owned edge: constants' cotangents
      const Vec<float> ca = S.cot(la), cb = S.cot(lb);
      gks += ms * (dotv(ca, us[0]) + dotv(cb, us[1]));
      if (hinge) {
        const Vec<float> cc = S.cot(lc), cd = S.cot(ld);
        gkb += mb * (dotv(ca, ub[0]) + dotv(cb, ub[1]) + dotv(cc, ub[2]) + dotv(cd, ub[3]));
      }
    }
  }
  __syncthreads();   // every edge slot written
  // faces, added to the slots of the edge each is attached to (an edge per
  // face: no two threads touch the same slot)
  for (int k = threadIdx.x; k < P.n_face; k += blockDim.x) {
    const uint2 fr = frec[k];
    const uint4 r = rec[fr.x & 0x3FFFFFFFu];
    const bool right = (fr.x >> 30) & 1u;
    const int la = r.x & 0xFFFF, lb = r.x >> 16;
    const int v0 = right ? lb : la, v1 = right ? la : lb;
    const int v2 = right ? (int)(r.y >> 16) : (int)(r.y & 0xFFFF);
    const int d0 = right ? (int)(r.z >> 16) : (int)(r.z & 0xFFFF);
    const int d1 = right ? (int)(r.z & 0xFFFF) : (int)(r.z >> 16);
    const int d2 = right ? (int)(r.w >> 16) : (int)(r.w & 0xFFFF);
    Vec<Dual> f[3], gA[3], gV[3], ua[3];
    float ea;
    const float ma = B.varied ? rest[5 * pe + pf + k] : 1.f;
    face_forces(S.pos(v0), S.pos(v1), S.pos(v2), rest[3 * pe + k], B.ka * ma, cA, cV, f, gA, gV,
                ua, ea);
    S.add(d0, f[0]);
    S.add(d1, f[1]);
    S.add(d2, f[2]);
    if (fr.x >> 31)
      gka += ma * (dotv(S.cot(v0), ua[0]) + dotv(S.cot(v1), ua[1]) + dotv(S.cot(v2), ua[2]));
  }
  __syncthreads();
  for (int i = threadIdx.x; i < P.n_own; i += blockDim.x) {
    const int s0 = ptr[i], s1 = ptr[i + 1];
    float jx = 0.f, jy = 0.f, jz = 0.f;
    for (int s = s0; s < s1; ++s) {
      jx += S.cx[s];
      jy += S.cy[s];
      jz += S.cz[s];
    }
    const int gvx = B.v_off + P.own0 + i;
    // traction part: the cotangents the faces left for this corner
    float wx = 0.f, wy = 0.f, wz = 0.f;   // the spread's velocity cotangent
    for (int q = vptr[i]; q < vptr[i + 1]; ++q) {
      const uint32_t e = vent[q];
      const int corner = (int)(e >> 30);
      const size_t gf = (size_t)B.f_off + (e & 0x3FFFFFFFu);
      jx += __ldg(T.gxe + (corner * 3 + 0) * (size_t)F + gf);
      jy += __ldg(T.gxe + (corner * 3 + 1) * (size_t)F + gf);
      jz += __ldg(T.gxe + (corner * 3 + 2) * (size_t)F + gf);
      if (gve) {
        wx += __ldg(gve + gf);
        wy += __ldg(gve + (size_t)F + gf);
        wz += __ldg(gve + 2 * (size_t)F + gf);
      }
    }
    const bool cl = T.clamp[gvx] != 0;
    const float gx0 = __ldg(gxn + gvx), gx1 = __ldg(gxn + V + gvx), gx2 = __ldg(gxn + 2 * V + gvx);
    gx[gvx] = gx0 + jx;
    gx[V + gvx] = gx1 + jy;
    gx[2 * V + gvx] = gx2 + jz;
    // a clamped node's new state does not depend on its velocity; the spread
    // (the centroid velocity of its faces) does
    gvo[gvx] = (cl ? 0.f : __ldg(gvn + gvx) + sc.dt * gx0) + wx;
    gvo[V + gvx] = (cl ? 0.f : __ldg(gvn + V + gvx) + sc.dt * gx1) + wy;
    gvo[2 * V + gvx] = (cl ? 0.f : __ldg(gvn + 2 * V + gvx) + sc.dt * gx2) + wz;
  }
  // constants' cotangents: fixed-order per-patch sums, then per body
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    gks += __shfl_down_sync(0xffffffffu, gks, o);
    gkb += __shfl_down_sync(0xffffffffu, gkb, o);
    gka += __shfl_down_sync(0xffffffffu, gka, o);
  }
  if ((threadIdx.x & 31) == 0) {
    s_red[0][threadIdx.x >> 5] = gks;
    s_red[1][threadIdx.x >> 5] = gkb;
    s_red[2][threadIdx.x >> 5] = gka;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (int k = 0; k < kForceThreads / 32; ++k) {
      a += s_red[0][k];
      b += s_red[1][k];
      c += s_red[2][k];
    }
    T.wpart[3 * (size_t)blockIdx.x] = a;
    T.wpart[3 * (size_t)blockIdx.x + 1] = b;
    T.wpart[3 * (size_t)blockIdx.x + 2] = c;
    __threadfence();
    s_last = (atomicAdd(T.wcounter + wk.x, 1) == topo.n_patch - 1);
  }
  __syncthreads();
  if (s_last && threadIdx.x == 0) {
    __threadfence();
    const volatile double* W = T.wpart;
    double a = 0.0, b = 0.0, c = 0.0;
    for (int k = 0; k < topo.n_patch; ++k) {
      a += W[3 * (size_t)(B.work_off + k)];
      b += W[3 * (size_t)(B.work_off + k) + 1];
      c += W[3 * (size_t)(B.work_off + k) + 2];
    }
    const double Ab = T.meas[2 * wk.x], Vb = T.meas[2 * wk.x + 1];
    gparams[5 * wk.x + 0] = a;
    gparams[5 * wk.x + 1] = b;
    gparams[5 * wk.x + 2] = c;
    gparams[5 * wk.x + 3] = -(Ab - B.A0) / B.A0 * dA;
    gparams[5 * wk.x + 4] = B.closed ? -(Vb - B.V0) / B.V0 * dV : 0.0;
    T.wcounter[wk.x] = 0;
  }
}

}  // namespace

cudaError_t launch_backward(ibm_ctx* c, const float* x, const float* v, const float* u,
                            const float* vv, const float* w, const float* pr, const float* accel,
                            const float* gx_next, const float* gv_next, const float* gfx,
                            const float* gfy, const float* gfz, float* gx, float* gv,
                            double* gparams) {
  if (c->n_chunks == 0) return cudaSuccess;
  // area, volume and the global-term coefficients at x
  cudaError_t e = zero_body_sums(c);
  if (e == cudaSuccess)
    e = launch_mls(c, x, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                   nullptr, nullptr, nullptr, nullptr, nullptr, true, false, false, false, false);
  if (e == cudaSuccess) e = launch_measure_finalize(c);
  if (e != cudaSuccess) return e;
  // per-face velocity cotangents of the spread go to the step's F_ext scratch,
  // unused by the adjoint otherwise
  float* gve = gfx ? c->d.fext : nullptr;
  ext_adjoint_kernel<<<c->n_chunks, kMT, 0, c->stream>>>(c->d, c->grid, c->sc, (int32_t)c->V,
                                                         (int32_t)c->F, x, v, u, vv, w, pr, accel,
                                                         gx_next, gv_next, gfx, gfy, gfz, gve);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  force_adjoint_kernel<<<c->n_work, kForceThreads, c->adjoint_smem, c->stream>>>(
      c->d, c->sc, (int32_t)c->V, (int32_t)c->F, x, gx_next, gv_next, gx, gv, gparams, gve);
  return cudaGetLastError();
}

cudaError_t set_adjoint_smem_limit(size_t bytes) {
  return cudaFuncSetAttribute(force_adjoint_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)bytes);
}

}  // namespace ibm
