// Taylor deformation of closed bodies and its adjoint (the drop measure of
// Sec. 3.1: semi-axes L and B of the deformed drop).
//
// The semi-axes are those of the ellipsoid with the same volume second
// moments: with V = sum of signed tetrahedra (origin, a, b, c), first moment
// m1 = sum V_t s/4 and second moment m2 = sum V_t/20 (sum_i p_i p_i^T + s s^T)
// (s = a + b + c, body frame), M = m2/V - ybar ybar^T, ybar = m1/V, the
// semi-axes are a_i = sqrt(5 lambda_i(M)) and D = (L - B)/(L + B) with L, B
// the largest and smallest.  Sums are float64 in a fixed order; the 3x3
// eigenproblem is solved per body by cyclic Jacobi rotations.
//
// The adjoint: dD/dlambda from D(L, B); dlambda_i/dM = v_i v_i^T (distinct
// eigenvalues); then back through M(m1, m2, V) and every face's tetrahedron.
#include <cuda_runtime.h>

#include "ibm_internal.cuh"

namespace ibm {
namespace {

// per face: V_t, m1 (3), m2 (xx, yy, zz, xy, xz, yz)
__device__ __forceinline__ void tet_moments(const double (&p1)[3], const double (&p2)[3],
                                            const double (&p3)[3], double (&m)[10]) {
  const double c[3] = {p2[1] * p3[2] - p2[2] * p3[1], p2[2] * p3[0] - p2[0] * p3[2],
                       p2[0] * p3[1] - p2[1] * p3[0]};
  const double Vt = (p1[0] * c[0] + p1[1] * c[1] + p1[2] * c[2]) / 6.0;
  const double s[3] = {p1[0] + p2[0] + p3[0], p1[1] + p2[1] + p3[1], p1[2] + p2[2] + p3[2]};
  m[0] = Vt;
  for (int d = 0; d < 3; ++d) m[1 + d] = Vt * s[d] / 4.0;
  const int I[6] = {0, 1, 2, 0, 0, 1}, J[6] = {0, 1, 2, 1, 2, 2};
  for (int q = 0; q < 6; ++q) {
    const int i = I[q], j = J[q];
    m[4 + q] = Vt / 20.0 * (p1[i] * p1[j] + p2[i] * p2[j] + p3[i] * p3[j] + s[i] * s[j]);
  }
}

// eigenvalues (ascending) and eigenvectors (columns) of a symmetric 3x3
__device__ void jacobi3(double (&A)[3][3], double (&lam)[3], double (&Vm)[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Vm[i][j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 30; ++sweep) {
    const double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
    const double dia = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
    if (off <= 1e-30 * dia || off == 0.0) break;
    for (int p = 0; p < 2; ++p)
      for (int q = p + 1; q < 3; ++q) {
        if (A[p][q] == 0.0) continue;
        // rotation that zeroes A[p][q]
        const double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
        for (int k = 0; k < 3; ++k) {
          const double akp = A[k][p], akq = A[k][q];
          A[k][p] = cs * akp - sn * akq;
          A[k][q] = sn * akp + cs * akq;
        }
        for (int k = 0; k < 3; ++k) {
          const double apk = A[p][k], aqk = A[q][k];
          A[p][k] = cs * apk - sn * aqk;
          A[q][k] = sn * apk + cs * aqk;
        }
        for (int k = 0; k < 3; ++k) {
          const double vkp = Vm[k][p], vkq = Vm[k][q];
          Vm[k][p] = cs * vkp - sn * vkq;
          Vm[k][q] = sn * vkp + cs * vkq;
        }
      }
  }
  int idx[3] = {0, 1, 2};
  for (int i = 0; i < 2; ++i)
    for (int j = i + 1; j < 3; ++j)
      if (A[idx[j]][idx[j]] < A[idx[i]][idx[i]]) {
        const int t = idx[i];
        idx[i] = idx[j];
        idx[j] = t;
      }
  double W[3][3];
  for (int i = 0; i < 3; ++i) {
    lam[i] = A[idx[i]][idx[i]];
    for (int k = 0; k < 3; ++k) W[k][i] = Vm[k][idx[i]];
  }
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) Vm[k][i] = W[k][i];
}

// one block per marker chunk: per-chunk moment partials; the last chunk of
// the body adds them in order and solves the eigenproblem
__global__ void __launch_bounds__(kMT) taylor_kernel(DeviceTables T, int32_t V,
                                                     const float* __restrict__ x,
                                                     double* __restrict__ D) {
  __shared__ double s_red[10][kMT / 32];
  __shared__ int s_last;
  const int4 ch = T.chunks[blockIdx.x];
  const BodyDev B = T.body[ch.x];
  const TopoDev topo = T.topo[B.topo];
  double m[10];
  for (int k = 0; k < 10; ++k) m[k] = 0.0;
  if ((int)threadIdx.x < ch.z && B.closed) {
    const int lf = __ldg(T.mface + topo.mface_off + ch.y + threadIdx.x);
    const int* tr = T.tri + topo.tri_off + 3 * lf;
    double p[3][3];
    for (int k = 0; k < 3; ++k) {
      const int gv = B.v_off + __ldg(tr + k);
      for (int d = 0; d < 3; ++d) p[k][d] = (double)__ldg(x + d * V + gv);
    }
    tet_moments(p[0], p[1], p[2], m);
  }
  for (int k = 0; k < 10; ++k) {
    double v = m[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_red[k][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  const int gc = B.chunk_off + ch.w;
  if (threadIdx.x < 10) {
    double v = 0.0;
    for (int w = 0; w < kMT / 32; ++w) v += s_red[threadIdx.x][w];
    T.tpart[10 * (size_t)gc + threadIdx.x] = v;
    __threadfence();   // every writer publishes its partial before the arrival count
  }
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(T.counter2 + ch.x, 1) == B.n_chunk - 1);
  __syncthreads();
  if (s_last && threadIdx.x == 0) {
    __threadfence();
    const volatile double* P = T.tpart;
    double t[10];
    for (int k = 0; k < 10; ++k) t[k] = 0.0;
    for (int c = 0; c < B.n_chunk; ++c)
      for (int k = 0; k < 10; ++k) t[k] += P[10 * (size_t)(B.chunk_off + c) + k];
    T.counter2[ch.x] = 0;
    double* out = T.taylor + 24 * (size_t)ch.x;
    for (int k = 0; k < 10; ++k) out[k] = t[k];
    if (!B.closed || !(t[0] > 0.0)) {
      D[ch.x] = 0.0;
      for (int k = 10; k < 24; ++k) out[k] = 0.0;
      return;
    }
    const double Vb = t[0];
    const double yb[3] = {t[1] / Vb, t[2] / Vb, t[3] / Vb};
    const double m2[3][3] = {{t[4], t[7], t[8]}, {t[7], t[5], t[9]}, {t[8], t[9], t[6]}};
    double M[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) M[i][j] = m2[i][j] / Vb - yb[i] * yb[j];
    double lam[3], Vm[3][3];
    jacobi3(M, lam, Vm);
    const double L = sqrt(5.0 * fmax(lam[2], 0.0)), Bm = sqrt(5.0 * fmax(lam[0], 0.0));
    D[ch.x] = (L - Bm) / (L + Bm);
    // keep what the adjoint needs: eigenvalues, eigenvectors of the extremes
    out[10] = lam[0];
    out[11] = lam[1];
    out[12] = lam[2];
    for (int k = 0; k < 3; ++k) {
      out[13 + k] = Vm[k][0];
      out[16 + k] = Vm[k][2];
    }
    out[19] = (lam[2] - lam[0]) / fmax(fabs(lam[2]), 1e-300);   // relative eigen-gap
  }
}

// per body: cotangents of V, m1, m2 from gD (one thread per body)
__global__ void taylor_body_adjoint(DeviceTables T, int32_t nb, const double* __restrict__ gD,
                                    double* __restrict__ gm) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const double* t = T.taylor + 24 * (size_t)b;
  double* o = gm + 10 * (size_t)b;
  for (int k = 0; k < 10; ++k) o[k] = 0.0;
  const double Vb = t[0];
  if (!(Vb > 0.0) || t[19] <= 0.0) return;
  const double L = sqrt(5.0 * t[12]), Bm = sqrt(5.0 * t[10]);
  const double s = (L + Bm) * (L + Bm);
  const double gL = gD[b] * 2.0 * Bm / s, gB = -gD[b] * 2.0 * L / s;
  const double glmax = gL * 5.0 / (2.0 * L), glmin = Bm > 0.0 ? gB * 5.0 / (2.0 * Bm) : 0.0;
  const double vmin[3] = {t[13], t[14], t[15]}, vmax[3] = {t[16], t[17], t[18]};
  double gM[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) gM[i][j] = glmax * vmax[i] * vmax[j] + glmin * vmin[i] * vmin[j];
  const double m1[3] = {t[1], t[2], t[3]};
  const double m2[3][3] = {{t[4], t[7], t[8]}, {t[7], t[5], t[9]}, {t[8], t[9], t[6]}};
  // M = m2/V - m1 m1^T / V^2
  double gV = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      gV += gM[i][j] * (-m2[i][j] / (Vb * Vb) + 2.0 * m1[i] * m1[j] / (Vb * Vb * Vb));
  o[0] = gV;
  for (int i = 0; i < 3; ++i) {
    double a = 0.0;
    for (int j = 0; j < 3; ++j) a += gM[i][j] * m1[j];
    o[1 + i] = -2.0 * a / (Vb * Vb);
  }
  // symmetric cotangent of m2 as (xx, yy, zz, xy, xz, yz) of gM / V
  o[4] = gM[0][0] / Vb;
  o[5] = gM[1][1] / Vb;
  o[6] = gM[2][2] / Vb;
  o[7] = gM[0][1] / Vb;
  o[8] = gM[0][2] / Vb;
  o[9] = gM[1][2] / Vb;
}

// per face: position cotangents of its tetrahedron, stored per corner
__global__ void __launch_bounds__(kMT) taylor_face_adjoint(DeviceTables T, int32_t V, int32_t F,
                                                           const float* __restrict__ x,
                                                           const double* __restrict__ gm) {
  const int4 ch = T.chunks[blockIdx.x];
  const BodyDev B = T.body[ch.x];
  const TopoDev topo = T.topo[B.topo];
  if ((int)threadIdx.x >= ch.z) return;
  const int lf = __ldg(T.mface + topo.mface_off + ch.y + threadIdx.x);
  const size_t gf = (size_t)B.f_off + lf;
  const double* g = gm + 10 * (size_t)ch.x;
  double gp[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  if (B.closed) {
    const int* tr = T.tri + topo.tri_off + 3 * lf;
    double p[3][3];
    for (int k = 0; k < 3; ++k) {
      const int gv = B.v_off + __ldg(tr + k);
      for (int d = 0; d < 3; ++d) p[k][d] = (double)__ldg(x + d * V + gv);
    }
    const double s[3] = {p[0][0] + p[1][0] + p[2][0], p[0][1] + p[1][1] + p[2][1],
                         p[0][2] + p[1][2] + p[2][2]};
    const double c23[3] = {p[1][1] * p[2][2] - p[1][2] * p[2][1], p[1][2] * p[2][0] - p[1][0] * p[2][2],
                           p[1][0] * p[2][1] - p[1][1] * p[2][0]};
    const double Vt = (p[0][0] * c23[0] + p[0][1] * c23[1] + p[0][2] * c23[2]) / 6.0;
    // full symmetric cotangent of m2
    const double G2[3][3] = {{g[4], g[7], g[8]}, {g[7], g[5], g[9]}, {g[8], g[9], g[6]}};
    double P[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        P[i][j] = p[0][i] * p[0][j] + p[1][i] * p[1][j] + p[2][i] * p[2][j] + s[i] * s[j];
    double gVt = g[0];
    for (int d = 0; d < 3; ++d) gVt += g[1 + d] * s[d] / 4.0;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) gVt += G2[i][j] * P[i][j] / 20.0;
    double gs[3];
    for (int i = 0; i < 3; ++i) {
      double a = 0.0;
      for (int j = 0; j < 3; ++j) a += 2.0 * G2[i][j] * s[j];
      gs[i] = Vt * g[1 + i] / 4.0 + Vt / 20.0 * a;
    }
    const double cr[3][3] = {{c23[0], c23[1], c23[2]},
                             {p[2][1] * p[0][2] - p[2][2] * p[0][1], p[2][2] * p[0][0] - p[2][0] * p[0][2],
                              p[2][0] * p[0][1] - p[2][1] * p[0][0]},
                             {p[0][1] * p[1][2] - p[0][2] * p[1][1], p[0][2] * p[1][0] - p[0][0] * p[1][2],
                              p[0][0] * p[1][1] - p[0][1] * p[1][0]}};
    for (int k = 0; k < 3; ++k)
      for (int i = 0; i < 3; ++i) {
        double a = 0.0;
        for (int j = 0; j < 3; ++j) a += 2.0 * G2[i][j] * p[k][j];
        gp[k][i] = Vt / 20.0 * a + gs[i] + gVt * cr[k][i] / 6.0;
      }
  }
  for (int k = 0; k < 3; ++k)
    for (int d = 0; d < 3; ++d) T.gxe[(k * 3 + d) * (size_t)F + gf] = (float)gp[k][d];
}

// per vertex: gather the corner cotangents of its faces (fixed order)
__global__ void __launch_bounds__(kForceThreads) corner_gather(DeviceTables T, int32_t V, int32_t F,
                                                              float* __restrict__ gx) {
  const int2 wk = T.work[blockIdx.x];
  const BodyDev B = T.body[wk.x];
  const TopoDev topo = T.topo[B.topo];
  const PatchHdr P = T.patch[topo.patch_off + wk.y];
  const int* tri = T.tri + topo.tri_off;
  const int* vp = T.v2f_ptr + topo.v2f_ptr_off;
  for (int i = threadIdx.x; i < P.n_own; i += blockDim.x) {
    const int lv = P.own0 + i;
    float a[3] = {0.f, 0.f, 0.f};
    for (int q = __ldg(vp + lv); q < __ldg(vp + lv + 1); ++q) {
      const int lf = __ldg(T.v2f_idx + topo.v2f_idx_off + q);
      const int corner = (__ldg(tri + 3 * lf) == lv) ? 0 : ((__ldg(tri + 3 * lf + 1) == lv) ? 1 : 2);
      const size_t gf = (size_t)B.f_off + lf;
      for (int d = 0; d < 3; ++d) a[d] += __ldg(T.gxe + (corner * 3 + d) * (size_t)F + gf);
    }
    const int gv = B.v_off + lv;
    for (int d = 0; d < 3; ++d) gx[d * V + gv] = a[d];
  }
}

}  // namespace

cudaError_t launch_taylor(ibm_ctx* c, const float* x, double* D) {
  if (c->n_chunks == 0) return cudaSuccess;
  taylor_kernel<<<c->n_chunks, kMT, 0, c->stream>>>(c->d, (int32_t)c->V, x, D);
  return cudaGetLastError();
}

cudaError_t launch_taylor_backward(ibm_ctx* c, const float* x, const double* gD, float* gx) {
  if (c->n_chunks == 0) return cudaSuccess;
  taylor_body_adjoint<<<(int)((c->B + 127) / 128), 128, 0, c->stream>>>(c->d, (int32_t)c->B, gD,
                                                                        c->d.tgrad);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  taylor_face_adjoint<<<c->n_chunks, kMT, 0, c->stream>>>(c->d, (int32_t)c->V, (int32_t)c->F, x,
                                                          c->d.tgrad);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  corner_gather<<<c->n_work, kForceThreads, 0, c->stream>>>(c->d, (int32_t)c->V, (int32_t)c->F, gx);
  return cudaGetLastError();
}

}  // namespace ibm
