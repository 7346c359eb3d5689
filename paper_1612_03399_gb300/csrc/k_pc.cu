// Strong coupling (Sec. 2.3): the elementwise parts of Hamming's fourth-order
// predictor-corrector for y = (x, v), y' = f(y) = (v, a(x)), and of the
// classical Runge-Kutta steps that start it.  The accelerations a(x) come
// from the marker and force kernels; these kernels only combine [3][V]
// arrays:
//   predictor  p = y_{n-3} + 4h/3 (2 f_n - f_{n-1} + 2 f_{n-2})
//   modifier   m = p - 112/121 (p_n - c_n)          (m = p on the first step)
//   corrector  c = (9 y_n - y_{n-2})/8 + 3h/8 (f(m) + 2 f_n - f_{n-1})
//   final      y_{n+1} = c + 9/121 (p - c),  and p - c is kept for the next step.
#include <cuda_runtime.h>

#include "ibm_internal.cuh"

namespace ibm {
namespace {

constexpr int kPcThreads = 256;

__global__ void __launch_bounds__(kPcThreads) lincomb_kernel(float* __restrict__ out, int64_t n,
                                                             LinComb L) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kLinCombMax; ++j)
      if (j < L.k) s = fmaf(L.c[j], __ldg(L.in[j] + i), s);
    out[i] = s;
  }
}

__global__ void __launch_bounds__(kPcThreads) ham_predict_kernel(HamPredict P, int64_t n) {
  const float q = 4.f * P.h / 3.f, mod = 112.f / 121.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float px = __ldg(P.x3 + i) + q * (2.f * __ldg(P.vn + i) - __ldg(P.vn1 + i) +
                                            2.f * __ldg(P.vn2 + i));
    const float pv = __ldg(P.v3 + i) + q * (2.f * __ldg(P.an + i) - __ldg(P.an1 + i) +
                                            2.f * __ldg(P.an2 + i));
    P.px[i] = px;
    P.pv[i] = pv;
    P.mx[i] = P.first ? px : px - mod * __ldg(P.pcx + i);
    P.mv[i] = P.first ? pv : pv - mod * __ldg(P.pcv + i);
  }
}

__global__ void __launch_bounds__(kPcThreads) ham_correct_kernel(HamCorrect C, int64_t n,
                                                                 int32_t V) {
  const float q = 3.f * C.h / 8.f, fin = 9.f / 121.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float xn = __ldg(C.xn + i), vn = __ldg(C.vn + i);
    const float cx = (9.f * xn - __ldg(C.x2 + i)) * 0.125f +
                     q * (__ldg(C.mv + i) + 2.f * vn - __ldg(C.vn1 + i));
    const float cv = (9.f * vn - __ldg(C.v2 + i)) * 0.125f +
                     q * (__ldg(C.am + i) + 2.f * __ldg(C.an + i) - __ldg(C.an1 + i));
    const float dx = __ldg(C.px + i) - cx, dv = __ldg(C.pv + i) - cv;
    const bool cl = C.clamp[i % V] != 0;   // clamped nodes keep x and have v = 0
    C.xo[i] = cl ? xn : cx + fin * dx;
    C.vo[i] = cl ? 0.f : cv + fin * dv;
    C.pcx[i] = cl ? 0.f : dx;
    C.pcv[i] = cl ? 0.f : dv;
  }
}

inline unsigned grid_for(int64_t n) {
  const int64_t b = (n + kPcThreads - 1) / kPcThreads;
  return (unsigned)(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

}  // namespace

cudaError_t launch_lincomb(ibm_ctx* c, float* out, const LinComb& L) {
  const int64_t n = 3 * c->V;
  if (n == 0) return cudaSuccess;
  lincomb_kernel<<<grid_for(n), kPcThreads, 0, c->stream>>>(out, n, L);
  return cudaGetLastError();
}

cudaError_t launch_ham_predict(ibm_ctx* c, const HamPredict& P) {
  const int64_t n = 3 * c->V;
  if (n == 0) return cudaSuccess;
  ham_predict_kernel<<<grid_for(n), kPcThreads, 0, c->stream>>>(P, n);
  return cudaGetLastError();
}

cudaError_t launch_ham_correct(ibm_ctx* c, const HamCorrect& C) {
  const int64_t n = 3 * c->V;
  if (n == 0) return cudaSuccess;
  ham_correct_kernel<<<grid_for(n), kPcThreads, 0, c->stream>>>(C, n, (int32_t)c->V);
  return cudaGetLastError();
}

}  // namespace ibm
