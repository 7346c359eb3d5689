// Element forces of the interaction potentials (Sec. 2.3, Eqs.
// elaspot..areapot), written once for any scalar type T: float in the forward
// force kernel, Dual (value + directional derivative) in the adjoint, where
// the derivative part of the forces is the Jacobian-vector product J y of
// the forces along the tangent y carried by the positions.  J = -Hessian of
// the energy is symmetric, so the same product is the vector-Jacobian
// product the adjoint needs.
//
// Edge e = (a, b) with wings c (face (a, b, c)) and d (face (b, a, d)):
//   spring   W = k_s/2 (l - l0)^2      F_a = k_s (l - l0) e/l, F_b = -F_a
//   bending  W = k_b (1 - cos(theta - theta0)),  F = -k_b sin(theta - theta0) grad theta,
//            cos theta = n1.n2, sin theta = (n1 x n2).e/|e|, and with
//            N1 = e x (c - a), N2 = (d - b) x e, s_c = (c - a).e/|e|^2, s_d likewise,
//            grad_c theta = -|e| N1/|N1|^2, grad_d theta = -|e| N2/|N2|^2,
//            grad_a theta = -(1 - s_c) grad_c - (1 - s_d) grad_d,
//            grad_b theta = -s_c grad_c - s_d grad_d
//            (the unique gradient that is invariant under translations and
//            rotations and moves the wings about the hinge).
// Face (a, b, c), A_f = |N|/2, n = N/|N|:
//   grad_a A_f = n x (c - b)/2 (cyclic), grad_a V = b x c / 6 (cyclic, body frame),
//   F = -(k_A (A - A0)/A0 + k_a (A_f - A0_f)/A0_f) grad A_f - k_v (V - V0)/V0 grad V.
#pragma once

#include <cuda_runtime.h>

namespace ibm {

// forward-mode dual number: value and derivative along one direction
struct Dual {
  float v, d;
  __device__ __forceinline__ Dual() {}
  __device__ __forceinline__ Dual(float a) : v(a), d(0.f) {}
  __device__ __forceinline__ Dual(float a, float b) : v(a), d(b) {}
};
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ Dual operator-(Dual a) { return {-a.v, -a.d}; }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.v * b.d + a.d * b.v}; }
__device__ __forceinline__ Dual operator/(Dual a, Dual b) {
  const float r = 1.f / b.v;
  const float q = a.v * r;
  return {q, (a.d - q * b.d) * r};
}
__device__ __forceinline__ float val(float a) { return a; }
__device__ __forceinline__ float val(Dual a) { return a.v; }
__device__ __forceinline__ float rsqrt_(float a) { return rsqrtf(a); }
__device__ __forceinline__ Dual rsqrt_(Dual a) {
  const float r = rsqrtf(a.v);
  return {r, -0.5f * r * r * r * a.d};
}

template <class T>
struct Vec {
  T x, y, z;
};
template <class T>
__device__ __forceinline__ Vec<T> vsub(const Vec<T>& a, const Vec<T>& b) {
  return {a.x - b.x, a.y - b.y, a.z - b.z};
}
template <class T>
__device__ __forceinline__ Vec<T> vadd(const Vec<T>& a, const Vec<T>& b) {
  return {a.x + b.x, a.y + b.y, a.z + b.z};
}
template <class T>
__device__ __forceinline__ Vec<T> vcross(const Vec<T>& a, const Vec<T>& b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <class T>
__device__ __forceinline__ T vdot(const Vec<T>& a, const Vec<T>& b) {
  return a.x * b.x + a.y * b.y + a.z * b.z;
}
template <class T>
__device__ __forceinline__ Vec<T> vscale(const Vec<T>& a, T s) {
  return {a.x * s, a.y * s, a.z * s};
}

// Spring and bending of one edge.  fa..fd receive the forces on a, b, c, d;
// `unit_s` and `unit_b` receive the same forces per unit k_s and k_b (for the
// constants' gradients); `has_hinge` false on a boundary edge.
template <class T>
__device__ __forceinline__ void edge_forces(const Vec<T>& pa, const Vec<T>& pb, const Vec<T>& pc,
                                            const Vec<T>& pd, bool has_hinge, float l0, float cos0,
                                            float sin0, float ks, float kb, Vec<T>& fa, Vec<T>& fb,
                                            Vec<T>& fc, Vec<T>& fd, Vec<T> (&unit_s)[2],
                                            Vec<T> (&unit_b)[4], float& e_spring, float& e_bend) {
  const Vec<T> e = vsub(pb, pa);
  const T l2 = vdot(e, e);
  const T inv_l = rsqrt_(l2);
  const T l = l2 * inv_l;
  const T s_unit = (l - T(l0)) * inv_l;
  unit_s[0] = vscale(e, s_unit);
  unit_s[1] = vscale(e, -s_unit);
  fa = vscale(unit_s[0], T(ks));
  fb = vscale(unit_s[1], T(ks));
  const float dl = val(l) - l0;
  e_spring = 0.5f * ks * dl * dl;
  const Vec<T> zero = {T(0.f), T(0.f), T(0.f)};
  fc = zero;
  fd = zero;
  e_bend = 0.f;
  if (!has_hinge) {
    unit_b[0] = unit_b[1] = unit_b[2] = unit_b[3] = zero;
    return;
  }
  const Vec<T> ac = vsub(pc, pa), ad = vsub(pd, pa);
  const Vec<T> N1 = vcross(e, ac);
  const Vec<T> N2 = vcross(vsub(pd, pb), e);
  const T q1 = vdot(N1, N1), q2 = vdot(N2, N2);
  const T r1 = rsqrt_(q1), r2 = rsqrt_(q2);
  const Vec<T> n1 = vscale(N1, r1), n2 = vscale(N2, r2);
  const T cth = vdot(n1, n2);
  const T sth = vdot(vcross(n1, n2), e) * inv_l;
  const T sdiff = sth * T(cos0) - cth * T(sin0);  // sin(theta - theta0)
  const Vec<T> gc = vscale(N1, -(l * r1 * r1));
  const Vec<T> gd = vscale(N2, -(l * r2 * r2));
  const T inv_l2 = inv_l * inv_l;
  const T sc = vdot(ac, e) * inv_l2, sd = vdot(ad, e) * inv_l2;
  const T one(1.f);
  const Vec<T> ga = vadd(vscale(gc, -(one - sc)), vscale(gd, -(one - sd)));
  const Vec<T> gb = vadd(vscale(gc, -sc), vscale(gd, -sd));
  const T cu = -sdiff;                 // force per unit k_b: -sin(theta - theta0) grad theta
  unit_b[0] = vscale(ga, cu);
  unit_b[1] = vscale(gb, cu);
  unit_b[2] = vscale(gc, cu);
  unit_b[3] = vscale(gd, cu);
  fa = vadd(fa, vscale(unit_b[0], T(kb)));
  fb = vadd(fb, vscale(unit_b[1], T(kb)));
  fc = vscale(unit_b[2], T(kb));
  fd = vscale(unit_b[3], T(kb));
  e_bend = kb * (1.f - (val(cth) * cos0 + val(sth) * sin0));
}

// Local area, global area and volume forces of one face.  cA, cV are the
// per-body coefficients k_A (A - A0)/A0 and k_v (V - V0)/V0 (as T, so that
// the adjoint can give them their directional derivative).  gradA, gradV
// receive grad A_f and grad V (body frame) at a, b, c; unit_a the force per
// unit k_a.
template <class T>
__device__ __forceinline__ void face_forces(const Vec<T>& pa, const Vec<T>& pb, const Vec<T>& pc,
                                            float A0f, float ka, T cA, T cV, Vec<T> (&f)[3],
                                            Vec<T> (&gradA)[3], Vec<T> (&gradV)[3],
                                            Vec<T> (&unit_a)[3], float& e_area) {
  const Vec<T> N = vcross(vsub(pb, pa), vsub(pc, pa));
  const T q = vdot(N, N);
  const T rn = rsqrt_(q);
  const T Af = T(0.5f) * q * rn;
  const Vec<T> n = vscale(N, rn);
  const T half(0.5f), sixth(1.f / 6.f);
  gradA[0] = vscale(vcross(n, vsub(pc, pb)), half);
  gradA[1] = vscale(vcross(n, vsub(pa, pc)), half);
  gradA[2] = vscale(vcross(n, vsub(pb, pa)), half);
  gradV[0] = vscale(vcross(pb, pc), sixth);
  gradV[1] = vscale(vcross(pc, pa), sixth);
  gradV[2] = vscale(vcross(pa, pb), sixth);
  const T strain = (Af - T(A0f)) / T(A0f);
  const T gA = cA + T(ka) * strain;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    unit_a[k] = vscale(gradA[k], -strain);
    f[k] = vadd(vscale(gradA[k], -gA), vscale(gradV[k], -cV));
  }
  const float da = val(Af) - A0f;
  e_area = 0.5f * ka * da * da / A0f;
}

}  // namespace ibm
