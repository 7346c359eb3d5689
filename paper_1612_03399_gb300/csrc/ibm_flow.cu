// The fluid phase (Sec. 2.1): incompressible Navier-Stokes on the triply
// periodic MAC grid with the three-substep RK3 fractional step.
//
// Per substep l:
//   rhs_kernel      H(u) (divergence form), and R = dt (gamma_l H + rho_l H_prev
//                   - alpha_l grad p + alpha_l nu lap u) for the three
//                   components, one thread per cell computing the u, v and w
//                   nodes of that cell index
//   the factorised Crank-Nicolson solve: the operator
//                   (1 - a d_xx)(1 - a d_yy)(1 - a d_zz), a = alpha_l dt nu / 2,
//                   is inverted in one of two exact ways, picked per substep
//                   at creation:
//     cn_solve_kernel  in real space: with c = a/h_d^2 the inverse of the
//                   periodic 1-D factor 1 - c (E - 2 + E^-1) is a circulant
//                   whose entries fall off as r^|m|, r < 1 the smaller root
//                   of c r^2 - (1 + 2c) r + c; when its mass beyond |m| = W
//                   (W <= 8) is below 2^-26 in every direction, the three
//                   inverses are applied as separable (2W+1)-tap filters and
//                   u* = u + du is written in the same pass
//     R2C (batch 3) -> cn_scale_kernel -> C2R, add_kernel (u* = u + du):
//                   otherwise, the operator being diagonal in Fourier space
//   div_kernel      div(u* + s f)
//   R2C -> poisson_scale_kernel -> C2R: lap(phi) = div / (alpha_l dt)
//   project_kernel  u = u* + s f - alpha_l dt grad(phi),
//                   p <- p + phi - a lap(phi)
// The eigenvalues of the periodic second difference, -(4/h^2) sin^2(pi k/n),
// are tabulated per direction in float64 on the host and stored as float.
#include <cuda_runtime.h>
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "ibm.h"
#include "ibm_internal.cuh"

struct ibm_flow {
  int device = 0;
  cudaStream_t stream = nullptr;
  int n[3] = {0, 0, 0};
  double L[3] = {0, 0, 0}, h[3] = {0, 0, 0};
  double nu = 0, dt = 0;
  size_t N = 0, NC = 0;         // cells; complex coefficients of one field
  float* H[2] = {nullptr, nullptr};   // [3][N] nonlinear terms, ping-pong
  int hcur = 0;                 // H[hcur] holds the last predictor's H(u)
  int last = -1;                // last predicted substep of the current step
  float* R = nullptr;           // [3][N] right-hand sides, then increments
  float* rp = nullptr;          // [N] divergence, then phi
  cufftComplex* S = nullptr;    // [3][NC] spectra
  float* lam = nullptr;         // [n_x/2 + 1 | n_y | n_z] eigenvalues
  cufftHandle r2c3 = 0, c2r3 = 0, r2c1 = 0, c2r1 = 0;
  bool plans = false;
  // per substep: the real-space solve's half width W (-1: Fourier path) and
  // its taps g[d][|m|] per direction, m = 0..W
  int solve_w[3] = {-1, -1, -1};
  float taps[3][3][9] = {};
  // phase timing (profiling aid): events at the 12 kernel boundaries of each
  // substep and the 3 of the body update
  bool timing = false;
  cudaEvent_t ev[3][12] = {};
  cudaEvent_t evs[3] = {};
  bool have_sub[3] = {false, false, false};
  bool have_struct = false;
};

namespace ibm {
namespace {

constexpr double kGamma[3] = {8.0 / 15.0, 5.0 / 12.0, 3.0 / 4.0};
constexpr double kRho[3] = {0.0, -17.0 / 60.0, -5.0 / 12.0};

struct FGrid {
  int nx, ny, nz;
  float ih[3], ih2[3];   // 1/h, 1/h^2
};

struct Vec3 {
  float* c[3];
};
struct CVec3 {
  const float* c[3];
};

// offsets of the six periodic neighbours of cell (i, j, k) relative to its
// index (grids below 2^31 cells, checked at creation): one 64-bit base per
// thread and 32-bit offsets instead of a full index per load
struct Nbr {
  int xp, xm, yp, ym, zp, zm;
  __device__ __forceinline__ Nbr(int i, int j, int k, int nx, int ny, int nz) {
    const int sxy = nx * ny;
    xp = i == nx - 1 ? 1 - nx : 1;
    xm = i == 0 ? nx - 1 : -1;
    yp = j == ny - 1 ? (1 - ny) * nx : nx;
    ym = j == 0 ? (ny - 1) * nx : -nx;
    zp = k == nz - 1 ? (1 - nz) * sxy : sxy;
    zm = k == 0 ? (nz - 1) * sxy : -sxy;
  }
};

// H(u) and the predictor's right-hand side at the u, v and w nodes of cell
// index (i, j, k).  Products for the d-derivative of component c are formed
// where the difference needs them: at the cell centres for d = c (mean of the
// two neighbouring c nodes, squared), at the (c, d) edges otherwise (mean of
// u_d along c times mean of u_c along d).
__global__ void __launch_bounds__(256) rhs_kernel(FGrid G, const float* __restrict__ u,
                                                  const float* __restrict__ v,
                                                  const float* __restrict__ w,
                                                  const float* __restrict__ p, CVec3 Hp, Vec3 Ho,
                                                  Vec3 Ro, float gam, float rho, float alpha,
                                                  float nu, float dt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= G.nx || j >= G.ny) return;
  const Nbr d(i, j, k, G.nx, G.ny, G.nz);
  const size_t o = ((size_t)k * G.ny + j) * G.nx + i;
  const float* up = u + o;
  const float* vp = v + o;
  const float* wp = w + o;
  const float* pp = p + o;
  const float U = __ldg(up), Uip = __ldg(up + d.xp), Uim = __ldg(up + d.xm),
              Ujp = __ldg(up + d.yp), Ujm = __ldg(up + d.ym), Ukp = __ldg(up + d.zp),
              Ukm = __ldg(up + d.zm), Uip_jm = __ldg(up + (d.xp + d.ym)),
              Uip_km = __ldg(up + (d.xp + d.zm));
  const float V = __ldg(vp), Vip = __ldg(vp + d.xp), Vim = __ldg(vp + d.xm),
              Vjp = __ldg(vp + d.yp), Vjm = __ldg(vp + d.ym), Vkp = __ldg(vp + d.zp),
              Vkm = __ldg(vp + d.zm), Vim_jp = __ldg(vp + (d.xm + d.yp)),
              Vjp_km = __ldg(vp + (d.yp + d.zm));
  const float W = __ldg(wp), Wip = __ldg(wp + d.xp), Wim = __ldg(wp + d.xm),
              Wjp = __ldg(wp + d.yp), Wjm = __ldg(wp + d.ym), Wkp = __ldg(wp + d.zp),
              Wkm = __ldg(wp + d.zm), Wim_kp = __ldg(wp + (d.xm + d.zp)),
              Wjm_kp = __ldg(wp + (d.ym + d.zp));
  const float P = __ldg(pp), Pim = __ldg(pp + d.xm), Pjm = __ldg(pp + d.ym),
              Pkm = __ldg(pp + d.zm);
  float H[3];
  {  // u nodes
    const float cp = 0.5f * (U + Uip), cm = 0.5f * (Uim + U);
    const float xx = (cp * cp - cm * cm) * G.ih[0];
    const float yy = (0.5f * (Vjp + Vim_jp) * 0.5f * (Ujp + U) - 0.5f * (V + Vim) * 0.5f * (U + Ujm)) * G.ih[1];
    const float zz = (0.5f * (Wkp + Wim_kp) * 0.5f * (Ukp + U) - 0.5f * (W + Wim) * 0.5f * (U + Ukm)) * G.ih[2];
    H[0] = -(xx + yy + zz);
  }
  {  // v nodes
    const float xx = (0.5f * (Uip + Uip_jm) * 0.5f * (Vip + V) - 0.5f * (U + Ujm) * 0.5f * (V + Vim)) * G.ih[0];
    const float cp = 0.5f * (V + Vjp), cm = 0.5f * (Vjm + V);
    const float yy = (cp * cp - cm * cm) * G.ih[1];
    const float zz = (0.5f * (Wkp + Wjm_kp) * 0.5f * (Vkp + V) - 0.5f * (W + Wjm) * 0.5f * (V + Vkm)) * G.ih[2];
    H[1] = -(xx + yy + zz);
  }
  {  // w nodes
    const float xx = (0.5f * (Uip + Uip_km) * 0.5f * (Wip + W) - 0.5f * (U + Ukm) * 0.5f * (W + Wim)) * G.ih[0];
    const float yy = (0.5f * (Vjp + Vjp_km) * 0.5f * (Wjp + W) - 0.5f * (V + Vkm) * 0.5f * (W + Wjm)) * G.ih[1];
    const float cp = 0.5f * (W + Wkp), cm = 0.5f * (Wkm + W);
    const float zz = (cp * cp - cm * cm) * G.ih[2];
    H[2] = -(xx + yy + zz);
  }
  const float Gp[3] = {(P - Pim) * G.ih[0], (P - Pjm) * G.ih[1], (P - Pkm) * G.ih[2]};
  const float Lu[3] = {
      (Uip - 2.f * U + Uim) * G.ih2[0] + (Ujp - 2.f * U + Ujm) * G.ih2[1] + (Ukp - 2.f * U + Ukm) * G.ih2[2],
      (Vip - 2.f * V + Vim) * G.ih2[0] + (Vjp - 2.f * V + Vjm) * G.ih2[1] + (Vkp - 2.f * V + Vkm) * G.ih2[2],
      (Wip - 2.f * W + Wim) * G.ih2[0] + (Wjp - 2.f * W + Wjm) * G.ih2[1] + (Wkp - 2.f * W + Wkm) * G.ih2[2]};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float r = gam * H[c] - alpha * Gp[c] + alpha * nu * Lu[c];
    if (Hp.c[c] != nullptr) r += rho * __ldg(Hp.c[c] + o);
    Ho.c[c][o] = H[c];
    Ro.c[c][o] = dt * r;
  }
}

// Spectra are [batch][nz][ny][nx/2+1]: one warp-wide row of x coefficients
// per threadIdx.y, rows (j, k) grid-strided over blockIdx.x, the batch in
// blockIdx.y (one division per row, none per coefficient).
constexpr int kRowThreads = 32, kRowsPerBlock = 8;

// times norm / prod_d (1 - a lam_d)
__global__ void __launch_bounds__(kRowThreads * kRowsPerBlock)
    cn_scale_kernel(cufftComplex* __restrict__ S, int nxh, int ny, int nz,
                    const float* __restrict__ lam, float a, float norm) {
  const float* lx = lam;
  const float* ly = lam + nxh;
  const float* lz = ly + ny;
  cufftComplex* Sb = S + (size_t)blockIdx.y * nz * ny * nxh;
  for (int r = blockIdx.x * kRowsPerBlock + threadIdx.y; r < ny * nz;
       r += gridDim.x * kRowsPerBlock) {
    const int k = r / ny, j = r - k * ny;
    const float dyz = norm / ((1.f - a * __ldg(ly + j)) * (1.f - a * __ldg(lz + k)));
    cufftComplex* row = Sb + (size_t)r * nxh;
    for (int i = threadIdx.x; i < nxh; i += kRowThreads) {
      const float s = dyz / (1.f - a * __ldg(lx + i));
      cufftComplex c = row[i];
      c.x *= s;
      c.y *= s;
      row[i] = c;
    }
  }
}

// spectrum of div / (alpha dt): times scale / (lam_x + lam_y + lam_z), mean 0
__global__ void __launch_bounds__(kRowThreads * kRowsPerBlock)
    poisson_scale_kernel(cufftComplex* __restrict__ S, int nxh, int ny, int nz,
                         const float* __restrict__ lam, float scale) {
  const float* lx = lam;
  const float* ly = lam + nxh;
  const float* lz = ly + ny;
  for (int r = blockIdx.x * kRowsPerBlock + threadIdx.y; r < ny * nz;
       r += gridDim.x * kRowsPerBlock) {
    const int k = r / ny, j = r - k * ny;
    const float lyz = __ldg(ly + j) + __ldg(lz + k);
    cufftComplex* row = S + (size_t)r * nxh;
    for (int i = threadIdx.x; i < nxh; i += kRowThreads) {
      const float l = __ldg(lx + i) + lyz;
      const float s = (r == 0 && i == 0) ? 0.f : scale / l;
      cufftComplex c = row[i];
      c.x *= s;
      c.y *= s;
      row[i] = c;
    }
  }
}

// u_c += du_c, du = [3][N]; the component in blockIdx.y
__global__ void add_kernel(Vec3 u, const float* __restrict__ du, size_t N) {
  const int c = blockIdx.y;
  float* uc = c == 0 ? u.c[0] : (c == 1 ? u.c[1] : u.c[2]);
  const float* dc = du + (size_t)c * N;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < N;
       q += (size_t)gridDim.x * blockDim.x)
    uc[q] += __ldg(dc + q);
}

// div(u* + s f) at the cell centres
__global__ void __launch_bounds__(256) div_kernel(FGrid G, CVec3 u, CVec3 f, float s,
                                                  float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= G.nx || j >= G.ny) return;
  const Nbr nb(i, j, k, G.nx, G.ny, G.nz);
  const size_t o = ((size_t)k * G.ny + j) * G.nx + i;
  const size_t oi = o + nb.xp, oj = o + nb.yp, ok = o + nb.zp;
  float d = (__ldg(u.c[0] + oi) - __ldg(u.c[0] + o)) * G.ih[0] +
            (__ldg(u.c[1] + oj) - __ldg(u.c[1] + o)) * G.ih[1] +
            (__ldg(u.c[2] + ok) - __ldg(u.c[2] + o)) * G.ih[2];
  if (f.c[0] != nullptr) {
    d += s * ((__ldg(f.c[0] + oi) - __ldg(f.c[0] + o)) * G.ih[0] +
              (__ldg(f.c[1] + oj) - __ldg(f.c[1] + o)) * G.ih[1] +
              (__ldg(f.c[2] + ok) - __ldg(f.c[2] + o)) * G.ih[2]);
  }
  out[o] = d;
}

// u = u* + s f - alpha dt grad(phi); p <- p + phi - a lap(phi)
__global__ void __launch_bounds__(256) project_kernel(FGrid G, Vec3 u, float* __restrict__ p,
                                                      const float* __restrict__ phi, CVec3 f,
                                                      float s, float adt, float a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= G.nx || j >= G.ny) return;
  const Nbr nb(i, j, k, G.nx, G.ny, G.nz);
  const size_t o = ((size_t)k * G.ny + j) * G.nx + i;
  const float* fp = phi + o;
  const float F = __ldg(fp);
  const float Fim = __ldg(fp + nb.xm), Fip = __ldg(fp + nb.xp);
  const float Fjm = __ldg(fp + nb.ym), Fjp = __ldg(fp + nb.yp);
  const float Fkm = __ldg(fp + nb.zm), Fkp = __ldg(fp + nb.zp);
  const float g[3] = {(F - Fim) * G.ih[0], (F - Fjm) * G.ih[1], (F - Fkm) * G.ih[2]};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float val = u.c[c][o] - adt * g[c];
    if (f.c[0] != nullptr) val += s * __ldg(f.c[c] + o);
    u.c[c][o] = val;
  }
  const float lap = (Fip - 2.f * F + Fim) * G.ih2[0] + (Fjp - 2.f * F + Fjm) * G.ih2[1] +
                    (Fkp - 2.f * F + Fkm) * G.ih2[2];
  p[o] += F - a * lap;
}

// asynchronous 4- and 8-byte global -> shared copies
__device__ __forceinline__ void cp_async4(float* sdst, const float* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async8(float* sdst, const float* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// The real-space factorised solve fused with u* = u + du.  A block owns a
// 32 x 32 tile of (x, y) outputs of one component over kSolveZ planes; it
// walks the kSolveZ + 2W planes that feed them (periodic wrap in every
// direction), each staged with its x and y halo by asynchronous copies two
// planes ahead.  Per plane: the x filter, four consecutive x per thread from
// float4 windows; the y filter for two x and two y per thread and the z
// filter in packed two-lane float arithmetic (pairs of x), from a register
// ring of the last 2W + 1 filtered planes; the z filter gives the output
// plane W planes back.  Taps are
// symmetric: g[d][|m|].
constexpr int kSolveT = 32, kSolveZ = 32, kMaxSolveW = 8;

struct SolveTaps {
  float g[3][kMaxSolveW + 1];
};
static_assert(sizeof(ibm_flow::taps[0]) == sizeof(SolveTaps), "tap table layout");

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

// symmetric filter of half width W centred on win[c]: g0 w_c + sum_m g_m (w_{c-m} + w_{c+m})
template <int W>
__device__ __forceinline__ float2 sym_filter(const float2* win, int c, const float* g) {
  float2 acc = __fmul2_rn(f2(g[0]), win[c]);
#pragma unroll
  for (int m = 1; m <= W; ++m) acc = __ffma2_rn(f2(g[m]), __fadd2_rn(win[c - m], win[c + m]), acc);
  return acc;
}

template <int W>
__global__ void __launch_bounds__(256, W <= 4 ? 3 : 2) cn_solve_kernel(FGrid G, const float* __restrict__ R,
                                                          Vec3 u, SolveTaps T) {
  constexpr int AY = kSolveT + 2 * W, AX = kSolveT + 2 * W;
  constexpr int NW4 = (4 + 2 * W + 3) / 4;          // float4s in an x window
  constexpr int AXP = kSolveT - 4 + 4 * NW4;        // row stride: windows stay in the row
  constexpr int AN = AY * AX, SLOTS = (AN + 255) / 256, NB = 3, NU = 4;
  static_assert(AXP >= AX && AXP % 4 == 0, "row stride");
  // dynamic shared memory: A[NB][AY * AXP] raw planes with halo,
  // Us[NU][32 * 32] u of the output planes, B[2][AY][32] x-filtered rows
  extern __shared__ __align__(16) float smem[];
  float (*A)[AY * AXP] = reinterpret_cast<float (*)[AY * AXP]>(smem);
  float (*Us)[kSolveT * kSolveT] = reinterpret_cast<float (*)[kSolveT * kSolveT]>(smem + NB * AY * AXP);
  float (*B)[AY][kSolveT] =
      reinterpret_cast<float (*)[AY][kSolveT]>(smem + NB * AY * AXP + NU * kSolveT * kSolveT);
  const int tid = threadIdx.x;
  const int nx = G.nx, ny = G.ny, nz = G.nz;
  const int ntx = (nx + kSolveT - 1) / kSolveT;
  const int x0 = (int)(blockIdx.y % ntx) * kSolveT, y0 = (int)(blockIdx.y / ntx) * kSolveT;
  const int k0 = (int)blockIdx.x * kSolveZ;
  const int nk = min(kSolveZ, nz - k0), nq = nk + 2 * W;
  const size_t plane = (size_t)nx * ny;
  const int c = blockIdx.z;
  const float* Rc = R + (size_t)c * plane * nz;
  float* uc = c == 0 ? u.c[0] : (c == 1 ? u.c[1] : u.c[2]);
  // staging slots: shared index and wrapped in-plane offset (-1 past the tile)
  int off[SLOTS];
  short sdst[SLOTS];
#pragma unroll
  for (int s = 0; s < SLOTS; ++s) {
    const int q = tid + 256 * s;
    off[s] = -1;
    sdst[s] = 0;
    if (q < AN) {
      const int r = q / AX, cc = q - r * AX;
      const int x = ((x0 - W + cc) % nx + nx) % nx, y = ((y0 - W + r) % ny + ny) % ny;
      off[s] = y * nx + x;
      sdst[s] = (short)(r * AXP + cc);
    }
  }
  // outputs: columns ox, ox + 1 of rows oy, oy + 1
  const int lx = (tid & 15) * 2, ly = (tid >> 4) * 2;
  const int ox = x0 + lx, oy = y0 + ly;
  // 8-byte aligned column pairs: even rows and an 8-byte aligned field
  const bool pair = (nx & 1) == 0 && (reinterpret_cast<uintptr_t>(uc) & 7) == 0;
  auto stage = [&](int q) {
    const int b = q % NB, bu = q % NU;
    int k = k0 - W + q;
    k = k < 0 ? k + nz : (k >= nz ? k - nz : k);
    const float* src = Rc + (size_t)k * plane;
#pragma unroll
    for (int s = 0; s < SLOTS; ++s)
      if (off[s] >= 0) cp_async4(&A[b][sdst[s]], src + off[s]);
    const int ko = q - 2 * W;
    if (ko >= 0) {
      const float* us = uc + (size_t)(k0 + ko) * plane;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        if (oy + j >= ny) continue;
        float* d = &Us[bu][(ly + j) * kSolveT + lx];
        const float* g = us + (size_t)(oy + j) * nx + ox;
        if (pair && ox + 1 < nx) {
          cp_async8(d, g);
        } else {
          if (ox < nx) cp_async4(d, g);
          if (ox + 1 < nx) cp_async4(d + 1, g + 1);
        }
      }
    }
    cp_async_commit();
  };
  float2 ring[2][2 * W + 1];
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int m = 0; m < 2 * W + 1; ++m) ring[j][m] = make_float2(0.f, 0.f);
  // x filter of plane q into B[q & 1]: item = (row, quad of four x)
  auto xfilter = [&](int q) {
    const float* a = A[q % NB];
    float (*Bq)[kSolveT] = B[q & 1];
    for (int it = tid; it < AY * 8; it += 256) {
      const int r = it >> 3, x4 = (it & 7) * 4;
      float win[4 * NW4];
      const float4* src = reinterpret_cast<const float4*>(a + r * AXP + x4);
#pragma unroll
      for (int v = 0; v < NW4; ++v) {
        const float4 t = src[v];
        win[4 * v] = t.x;
        win[4 * v + 1] = t.y;
        win[4 * v + 2] = t.z;
        win[4 * v + 3] = t.w;
      }
      float o[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float acc = T.g[0][0] * win[j + W];
#pragma unroll
        for (int m = 1; m <= W; ++m) acc += T.g[0][m] * (win[j + W - m] + win[j + W + m]);
        o[j] = acc;
      }
      *reinterpret_cast<float4*>(&Bq[r][x4]) = make_float4(o[0], o[1], o[2], o[3]);
    }
  };
  // one barrier per plane: the y and z filters of plane q and the x filter
  // of plane q + 1 run between two barriers (B double-buffered, A three
  // planes, Us four)
  stage(0);
  if (nq > 1) stage(1);
  if (nq > 1)
    cp_async_wait<1>();
  else
    cp_async_wait<0>();
  __syncthreads();
  if (nq > 2) stage(2);
  xfilter(0);
  for (int q = 0; q < nq; ++q) {
    if (q + 2 < nq)
      cp_async_wait<1>();
    else
      cp_async_wait<0>();
    // B[q & 1] complete and plane q + 1 visible; every thread is past the x
    // filter of plane q (A[q % NB] free) and the y filter of plane q - 1
    // (B[(q + 1) & 1] and Us[(q - 1) % NU] free)
    __syncthreads();
    if (q + 3 < nq) stage(q + 3);
    // y filter: rows ly, ly + 1 of columns lx, lx + 1
    {
      float2 col[2 + 2 * W];
#pragma unroll
      for (int i = 0; i < 2 + 2 * W; ++i)
        col[i] = *reinterpret_cast<const float2*>(&B[q & 1][ly + i][lx]);
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const float2 v = sym_filter<W>(col, j + W, T.g[1]);
#pragma unroll
        for (int m = 0; m < 2 * W; ++m) ring[j][m] = ring[j][m + 1];
        ring[j][2 * W] = v;
      }
    }
    const int ko = q - 2 * W;
    if (ko >= 0) {
      float* uo = uc + (size_t)(k0 + ko) * plane;
      const float* ub = Us[q % NU];
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        if (oy + j >= ny) continue;
        const float2 d = sym_filter<W>(ring[j], W, T.g[2]);
        const float2 uu = *reinterpret_cast<const float2*>(&ub[(ly + j) * kSolveT + lx]);
        const float2 r = __fadd2_rn(uu, d);
        float* g = uo + (size_t)(oy + j) * nx + ox;
        if (pair && ox + 1 < nx) {
          *reinterpret_cast<float2*>(g) = r;
        } else {
          if (ox < nx) g[0] = r.x;
          if (ox + 1 < nx) g[1] = r.y;
        }
      }
    }
    if (q + 1 < nq) xfilter(q + 1);
  }
}

// dynamic shared memory of cn_solve_kernel<W>
constexpr size_t solve_smem(int W) {
  return sizeof(float) * (3 * (size_t)(kSolveT + 2 * W) * (kSolveT - 4 + 4 * ((4 + 2 * W + 3) / 4)) +
                          4 * (size_t)kSolveT * kSolveT + 2 * (size_t)(kSolveT + 2 * W) * kSolveT);
}

// allow each real-space substep's kernel its dynamic shared memory
cudaError_t set_solve_smem(const ibm_flow* fl) {
  cudaError_t e = cudaSuccess;
  for (int l = 0; l < 3 && e == cudaSuccess; ++l) {
    switch (fl->solve_w[l]) {
#define IBM_SOLVE_ATTR(WW)                                                                 \
  case WW:                                                                                 \
    e = cudaFuncSetAttribute(cn_solve_kernel<WW>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             (int)solve_smem(WW));                                         \
    break;
      IBM_SOLVE_ATTR(0) IBM_SOLVE_ATTR(1) IBM_SOLVE_ATTR(2) IBM_SOLVE_ATTR(3) IBM_SOLVE_ATTR(4)
      IBM_SOLVE_ATTR(5) IBM_SOLVE_ATTR(6) IBM_SOLVE_ATTR(7) IBM_SOLVE_ATTR(8)
#undef IBM_SOLVE_ATTR
      default: break;
    }
  }
  return e;
}

FGrid fgrid(const ibm_flow* fl);

cudaError_t launch_cn_solve(const ibm_flow* fl, int l, float* u, float* v, float* w,
                            cudaStream_t s) {
  const FGrid G = fgrid(fl);
  SolveTaps T;
  for (int d = 0; d < 3; ++d)
    for (int m = 0; m <= kMaxSolveW; ++m) T.g[d][m] = fl->taps[l][d][m];
  const unsigned tiles = (unsigned)(((fl->n[0] + kSolveT - 1) / kSolveT) *
                                    ((fl->n[1] + kSolveT - 1) / kSolveT));
  const dim3 grid((unsigned)((fl->n[2] + kSolveZ - 1) / kSolveZ), tiles, 3), block(256);
  const Vec3 U{{u, v, w}};
  switch (fl->solve_w[l]) {
#define IBM_SOLVE_CASE(WW) \
  case WW: cn_solve_kernel<WW><<<grid, block, solve_smem(WW), s>>>(G, fl->R, U, T); break;
    IBM_SOLVE_CASE(0) IBM_SOLVE_CASE(1) IBM_SOLVE_CASE(2) IBM_SOLVE_CASE(3) IBM_SOLVE_CASE(4)
    IBM_SOLVE_CASE(5) IBM_SOLVE_CASE(6) IBM_SOLVE_CASE(7) IBM_SOLVE_CASE(8)
#undef IBM_SOLVE_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

FGrid fgrid(const ibm_flow* fl) {
  FGrid G;
  G.nx = fl->n[0];
  G.ny = fl->n[1];
  G.nz = fl->n[2];
  for (int d = 0; d < 3; ++d) {
    G.ih[d] = (float)(1.0 / fl->h[d]);
    G.ih2[d] = (float)(1.0 / (fl->h[d] * fl->h[d]));
  }
  return G;
}

dim3 cell_grid(const ibm_flow* fl) {
  return dim3((unsigned)((fl->n[0] + 31) / 32), (unsigned)((fl->n[1] + 7) / 8), (unsigned)fl->n[2]);
}

// blocks for the row kernels: enough rows in flight, at most one pass over them
unsigned row_blocks(const ibm_flow* fl) {
  const int rows = fl->n[1] * fl->n[2];
  const int b = (rows + kRowsPerBlock - 1) / kRowsPerBlock;
  return (unsigned)(b < 152 * 32 ? b : 152 * 32);
}

unsigned flat_blocks(size_t total) {
  const size_t b = (total + 255) / 256;
  return (unsigned)(b < (size_t)152 * 16 ? (b > 0 ? b : 1) : (size_t)152 * 16);
}

cudaError_t fft_status(cufftResult r) {
  return r == CUFFT_SUCCESS ? cudaSuccess : cudaErrorUnknown;
}

cudaError_t set_plan_streams(ibm_flow* fl, cudaStream_t s) {
  for (cufftHandle h : {fl->r2c3, fl->c2r3, fl->r2c1, fl->c2r1})
    if (cufftSetStream(h, s) != CUFFT_SUCCESS) return cudaErrorUnknown;
  return cudaSuccess;
}

void release(ibm_flow* fl) {
  if (fl->plans) {
    cufftDestroy(fl->r2c3);
    cufftDestroy(fl->c2r3);
    cufftDestroy(fl->r2c1);
    cufftDestroy(fl->c2r1);
  }
  for (void* q : {(void*)fl->H[0], (void*)fl->H[1], (void*)fl->R, (void*)fl->rp, (void*)fl->S,
                  (void*)fl->lam})
    if (q) cudaFree(q);
  for (auto& row : fl->ev)
    for (cudaEvent_t& ev : row)
      if (ev) cudaEventDestroy(ev);
  for (cudaEvent_t& ev : fl->evs)
    if (ev) cudaEventDestroy(ev);
}

// Entries g_m, m = 0..kMaxSolveW, of the inverse of the periodic n-point
// operator 1 - c (E - 2 + E^-1): its eigenvalues are 1 + 4c sin^2(pi k/n), so
// g_m = (1/n) sum_k cos(2 pi k m/n) / (1 + 4c sin^2(pi k/n))  (float64).
// They are positive and sum to 1 over a period.
void inverse_taps(double cc, int n, double* g) {
  for (int m = 0; m <= kMaxSolveW; ++m) {
    double acc = 0.0;
    for (int k = 0; k < n; ++k) {
      const double sn = std::sin(M_PI * k / n);
      acc += std::cos(2.0 * M_PI * (double)k * m / n) / (1.0 + 4.0 * cc * sn * sn);
    }
    g[m] = acc / n;
  }
}

// Picks each substep's solve: the smallest W <= kMaxSolveW, 2W + 1 <= n_d,
// with the mass of the entries beyond |m| = W below 2^-26 in every
// direction (real space), else the Fourier path (W = -1; also for planes of
// more than 65535 tiles).
void choose_solves(ibm_flow* fl) {
  const long tiles = (long)((fl->n[0] + kSolveT - 1) / kSolveT) * ((fl->n[1] + kSolveT - 1) / kSolveT);
  for (int l = 0; l < 3; ++l) {
    if (tiles > 65535) {   // the launch's grid.y
      fl->solve_w[l] = -1;
      continue;
    }
    const double a = (kGamma[l] + kRho[l]) * fl->dt * fl->nu / 2.0;
    int wl = 0;
    double g[3][kMaxSolveW + 1];
    for (int d = 0; d < 3 && wl >= 0; ++d) {
      inverse_taps(a / (fl->h[d] * fl->h[d]), fl->n[d], g[d]);
      int wd = -1;
      double inner = g[d][0];
      for (int w = 0; w <= kMaxSolveW && 2 * w + 1 <= fl->n[d]; ++w) {
        if (w > 0) inner += 2.0 * g[d][w];
        if (1.0 - inner <= std::ldexp(1.0, -26)) {
          wd = w;
          break;
        }
      }
      wl = wd < 0 ? -1 : std::max(wl, wd);
    }
    fl->solve_w[l] = wl;
    for (int d = 0; d < 3; ++d)
      for (int m = 0; m <= kMaxSolveW; ++m)
        fl->taps[l][d][m] = wl >= 0 && m <= wl ? (float)g[d][m] : 0.f;
  }
}

ibm_status flow_err(ibm_status s, const std::string& m) {
  set_global_error(m);
  return s;
}

}  // namespace

// record boundary k of substep l (k = 0..11) when phase timing is on
cudaError_t flow_mark(ibm_flow* fl, int l, int k, cudaStream_t s) {
  if (!fl->timing) return cudaSuccess;
  return cudaEventRecord(fl->ev[l][k], s);
}

// record boundary k (0..2) of the body update: its start, after the marker
// kernel (body sums and probe traction), after the force kernel
cudaError_t flow_mark_struct(ibm_flow* fl, int k, cudaStream_t s) {
  if (!fl->timing) return cudaSuccess;
  const cudaError_t e = cudaEventRecord(fl->evs[k], s);
  if (e == cudaSuccess && k == 2) fl->have_struct = true;
  return e;
}

cudaError_t flow_predict(ibm_flow* fl, int l, float* u, float* v, float* w, const float* p,
                         cudaStream_t s) {
  const FGrid G = fgrid(fl);
  const float dt = (float)fl->dt, nu = (float)fl->nu;
  const double alpha = kGamma[l] + kRho[l];
  CVec3 Hp{{nullptr, nullptr, nullptr}};
  if (kRho[l] != 0.0)
    for (int c = 0; c < 3; ++c) Hp.c[c] = fl->H[fl->hcur] + c * fl->N;
  float* Hn = fl->H[fl->hcur ^ 1];
  const Vec3 Ho{{Hn, Hn + fl->N, Hn + 2 * fl->N}};
  const Vec3 Ro{{fl->R, fl->R + fl->N, fl->R + 2 * fl->N}};
  cudaError_t e = set_plan_streams(fl, s);
  if (e != cudaSuccess) return e;
  e = flow_mark(fl, l, 0, s);
  if (e != cudaSuccess) return e;
  rhs_kernel<<<cell_grid(fl), dim3(32, 8), 0, s>>>(G, u, v, w, p, Hp, Ho, Ro, (float)kGamma[l],
                                                     (float)kRho[l], (float)alpha, nu, dt);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = flow_mark(fl, l, 1, s);
  const bool fourier = fl->solve_w[l] < 0;
  // real-space path: the three Fourier phases stay empty
  if (e == cudaSuccess && fourier) e = fft_status(cufftExecR2C(fl->r2c3, fl->R, fl->S));
  if (e == cudaSuccess) e = flow_mark(fl, l, 2, s);
  if (e == cudaSuccess && fourier) {
    const int nxh = fl->n[0] / 2 + 1;
    cn_scale_kernel<<<dim3(row_blocks(fl), 3), dim3(kRowThreads, kRowsPerBlock), 0, s>>>(
        fl->S, nxh, fl->n[1], fl->n[2], fl->lam, (float)(alpha * fl->dt * fl->nu / 2.0),
        (float)(1.0 / (double)fl->N));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = flow_mark(fl, l, 3, s);
  if (e == cudaSuccess && fourier) e = fft_status(cufftExecC2R(fl->c2r3, fl->S, fl->R));
  if (e == cudaSuccess) e = flow_mark(fl, l, 4, s);
  if (e == cudaSuccess && fourier) {
    add_kernel<<<dim3(flat_blocks(fl->N), 3), 256, 0, s>>>(Vec3{{u, v, w}}, fl->R, fl->N);
    e = cudaGetLastError();
  } else if (e == cudaSuccess) {
    e = launch_cn_solve(fl, l, u, v, w, s);
  }
  if (e == cudaSuccess) e = flow_mark(fl, l, 5, s);
  if (e == cudaSuccess) {
    fl->hcur ^= 1;
    fl->last = l;
  }
  return e;
}

cudaError_t flow_project(ibm_flow* fl, int l, float* u, float* v, float* w, float* p,
                         const float* fx, const float* fy, const float* fz, float fscale,
                         cudaStream_t s) {
  const FGrid G = fgrid(fl);
  const double alpha = kGamma[l] + kRho[l];
  const CVec3 f{{fx, fy, fz}};
  cudaError_t e = set_plan_streams(fl, s);
  if (e != cudaSuccess) return e;
  e = flow_mark(fl, l, 6, s);
  if (e != cudaSuccess) return e;
  div_kernel<<<cell_grid(fl), dim3(32, 8), 0, s>>>(G, CVec3{{u, v, w}}, f, fscale, fl->rp);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = flow_mark(fl, l, 7, s);
  if (e == cudaSuccess) e = fft_status(cufftExecR2C(fl->r2c1, fl->rp, fl->S));
  if (e == cudaSuccess) e = flow_mark(fl, l, 8, s);
  if (e == cudaSuccess) {
    const int nxh = fl->n[0] / 2 + 1;
    poisson_scale_kernel<<<row_blocks(fl), dim3(kRowThreads, kRowsPerBlock), 0, s>>>(
        fl->S, nxh, fl->n[1], fl->n[2], fl->lam, (float)(1.0 / ((double)fl->N * alpha * fl->dt)));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = flow_mark(fl, l, 9, s);
  if (e == cudaSuccess) e = fft_status(cufftExecC2R(fl->c2r1, fl->S, fl->rp));
  if (e == cudaSuccess) e = flow_mark(fl, l, 10, s);
  if (e == cudaSuccess) {
    project_kernel<<<cell_grid(fl), dim3(32, 8), 0, s>>>(
        G, Vec3{{u, v, w}}, p, fl->rp, f, fscale, (float)(alpha * fl->dt),
        (float)(alpha * fl->dt * fl->nu / 2.0));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = flow_mark(fl, l, 11, s);
  if (e == cudaSuccess && fl->timing) fl->have_sub[l] = true;
  return e;
}

bool flow_matches(const ibm_flow* fl, const ibm_grid_desc& g, double dt, double mu) {
  for (int d = 0; d < 3; ++d)
    if (g.n[d] != fl->n[d] || std::fabs(g.L[d] - fl->L[d]) > 1e-12 * std::fabs(fl->L[d]))
      return false;
  return std::fabs(dt - fl->dt) <= 1e-12 * fl->dt && std::fabs(mu - fl->nu) <= 1e-12 * (1.0 + fl->nu);
}

cudaStream_t flow_stream(const ibm_flow* fl) { return fl->stream; }
int flow_device(const ibm_flow* fl) { return fl->device; }
size_t flow_cells(const ibm_flow* fl) { return fl->N; }

}  // namespace ibm

using ibm::flow_err;

extern "C" ibm_status ibm_flow_create(const ibm_grid_desc* grid, double nu, double dt,
                                      ibm_flow** out) {
  if (out) *out = nullptr;
  if (!grid || !out) return flow_err(IBM_ERR_INVALID_ARG, "ibm_flow_create: null argument");
  for (int d = 0; d < 3; ++d)
    if (grid->n[d] < 4 || !(grid->L[d] > 0.0) || !std::isfinite(grid->L[d]))
      return flow_err(IBM_ERR_INVALID_ARG, "ibm_flow_create: grid needs n >= 4 and L > 0");
  if ((double)grid->n[0] * grid->n[1] * grid->n[2] >= 2147483648.0)
    return flow_err(IBM_ERR_UNSUPPORTED, "ibm_flow_create: grids of 2^31 cells or more");
  if (grid->n[2] > 65535 || (grid->n[1] + 7) / 8 > 65535)
    return flow_err(IBM_ERR_UNSUPPORTED, "ibm_flow_create: n_z above 65535 or n_y above 524280");
  if (!(nu >= 0.0) || !std::isfinite(nu) || !(dt > 0.0) || !std::isfinite(dt))
    return flow_err(IBM_ERR_INVALID_ARG, "ibm_flow_create: needs nu >= 0 and dt > 0");
  ibm_flow* fl = new ibm_flow();
  cudaGetDevice(&fl->device);
  for (int d = 0; d < 3; ++d) {
    fl->n[d] = grid->n[d];
    fl->L[d] = grid->L[d];
    fl->h[d] = grid->L[d] / grid->n[d];
  }
  fl->nu = nu;
  fl->dt = dt;
  ibm::choose_solves(fl);
  const int nx = fl->n[0], ny = fl->n[1], nz = fl->n[2], nxh = nx / 2 + 1;
  fl->N = (size_t)nx * ny * nz;
  fl->NC = (size_t)nxh * ny * nz;
  cudaError_t e = cudaSuccess;
  e = ibm::set_solve_smem(fl);
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = cudaMalloc(&fl->H[b], 3 * fl->N * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&fl->R, 3 * fl->N * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&fl->rp, fl->N * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&fl->S, 3 * fl->NC * sizeof(cufftComplex));
  if (e == cudaSuccess) e = cudaMalloc(&fl->lam, (size_t)(nxh + ny + nz) * sizeof(float));
  if (e == cudaSuccess) {
    std::vector<float> lam;
    const int m[3] = {nxh, ny, nz};
    for (int d = 0; d < 3; ++d)
      for (int q = 0; q < m[d]; ++q) {
        const double s = std::sin(M_PI * q / fl->n[d]);
        lam.push_back((float)(-(4.0 / (fl->h[d] * fl->h[d])) * s * s));
      }
    e = cudaMemcpy(fl->lam, lam.data(), lam.size() * sizeof(float), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    ibm::release(fl);
    delete fl;
    cudaGetLastError();
    return flow_err(e == cudaErrorMemoryAllocation ? IBM_ERR_OOM : IBM_ERR_CUDA,
                    std::string("ibm_flow_create: ") + cudaGetErrorString(e));
  }
  int dims[3] = {nz, ny, nx};
  cufftResult r = cufftPlanMany(&fl->r2c3, 3, dims, nullptr, 1, 0, nullptr, 1, 0, CUFFT_R2C, 3);
  bool ok = r == CUFFT_SUCCESS;
  if (ok) ok = cufftPlanMany(&fl->c2r3, 3, dims, nullptr, 1, 0, nullptr, 1, 0, CUFFT_C2R, 3) == CUFFT_SUCCESS;
  if (ok) ok = cufftPlan3d(&fl->r2c1, nz, ny, nx, CUFFT_R2C) == CUFFT_SUCCESS;
  if (ok) ok = cufftPlan3d(&fl->c2r1, nz, ny, nx, CUFFT_C2R) == CUFFT_SUCCESS;
  if (!ok) {
    // plans created so far are destroyed individually
    for (cufftHandle h : {fl->r2c3, fl->c2r3, fl->r2c1, fl->c2r1})
      if (h) cufftDestroy(h);
    fl->plans = false;
    ibm::release(fl);
    delete fl;
    return flow_err(IBM_ERR_CUDA, "ibm_flow_create: cuFFT plan creation failed");
  }
  fl->plans = true;
  *out = fl;
  return IBM_OK;
}

extern "C" ibm_status ibm_flow_solve_width(const ibm_flow* fl, int32_t substep, int32_t* width) {
  if (!fl || !width) return flow_err(IBM_ERR_INVALID_ARG, "ibm_flow_solve_width: null argument");
  if (substep < 0 || substep > 2)
    return flow_err(IBM_ERR_INVALID_ARG, "ibm_flow_solve_width: substep must be 0, 1 or 2");
  *width = fl->solve_w[substep];
  return IBM_OK;
}

extern "C" ibm_status ibm_flow_set_stream(ibm_flow* fl, void* stream) {
  if (!fl) return flow_err(IBM_ERR_INVALID_ARG, "ibm_flow_set_stream: null flow");
  fl->stream = static_cast<cudaStream_t>(stream);
  return IBM_OK;
}

extern "C" void ibm_flow_destroy(ibm_flow* fl) {
  if (!fl) return;
  cudaSetDevice(fl->device);
  // coupled steps run on a context's stream: wait for all work on the device
  cudaDeviceSynchronize();
  ibm::release(fl);
  delete fl;
}

extern "C" ibm_status ibm_flow_predict(ibm_flow* fl, int32_t substep, float* u, float* v,
                                       float* w, const float* p) {
  if (!fl || !u || !v || !w || !p) return flow_err(IBM_ERR_INVALID_ARG, "ibm_flow_predict: null argument");
  if (substep < 0 || substep > 2)
    return flow_err(IBM_ERR_INVALID_ARG, "ibm_flow_predict: substep must be 0, 1 or 2");
  if (substep > 0 && fl->last != substep - 1)
    return flow_err(IBM_ERR_INVALID_ARG, "ibm_flow_predict: substeps must run in order");
  cudaSetDevice(fl->device);
  const cudaError_t e = ibm::flow_predict(fl, substep, u, v, w, p, fl->stream);
  if (e != cudaSuccess)
    return flow_err(IBM_ERR_CUDA, std::string("ibm_flow_predict: ") + cudaGetErrorString(e));
  return IBM_OK;
}

extern "C" ibm_status ibm_flow_project(ibm_flow* fl, int32_t substep, float* u, float* v,
                                       float* w, float* p, const float* fx, const float* fy,
                                       const float* fz, float f_scale) {
  if (!fl || !u || !v || !w || !p) return flow_err(IBM_ERR_INVALID_ARG, "ibm_flow_project: null argument");
  if (substep < 0 || substep > 2)
    return flow_err(IBM_ERR_INVALID_ARG, "ibm_flow_project: substep must be 0, 1 or 2");
  const bool any = fx || fy || fz;
  if (any && !(fx && fy && fz))
    return flow_err(IBM_ERR_INVALID_ARG, "ibm_flow_project: give all three force fields or none");
  cudaSetDevice(fl->device);
  const cudaError_t e = ibm::flow_project(fl, substep, u, v, w, p, fx, fy, fz, f_scale, fl->stream);
  if (e != cudaSuccess)
    return flow_err(IBM_ERR_CUDA, std::string("ibm_flow_project: ") + cudaGetErrorString(e));
  return IBM_OK;
}

extern "C" ibm_status ibm_flow_set_phase_timing(ibm_flow* fl, int32_t on) {
  if (!fl) return flow_err(IBM_ERR_INVALID_ARG, "ibm_flow_set_phase_timing: null flow");
  cudaSetDevice(fl->device);
  if (on && !fl->ev[0][0]) {
    for (auto& row : fl->ev)
      for (cudaEvent_t& ev : row) {
        const cudaError_t e = cudaEventCreate(&ev);
        if (e != cudaSuccess)
          return flow_err(IBM_ERR_CUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(e));
      }
    for (cudaEvent_t& ev : fl->evs) {
      const cudaError_t e = cudaEventCreate(&ev);
      if (e != cudaSuccess)
        return flow_err(IBM_ERR_CUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(e));
    }
  }
  fl->timing = on != 0;
  for (bool& b : fl->have_sub) b = false;
  fl->have_struct = false;
  return IBM_OK;
}

extern "C" ibm_status ibm_flow_get_phase_times(ibm_flow* fl, float* ms) {
  if (!fl || !ms) return flow_err(IBM_ERR_INVALID_ARG, "ibm_flow_get_phase_times: null argument");
  for (bool b : fl->have_sub)
    if (!b)
      return flow_err(IBM_ERR_INVALID_ARG,
                      "ibm_flow_get_phase_times: no timed substep 0, 1 and 2 recorded");
  cudaSetDevice(fl->device);
  cudaError_t e = cudaEventSynchronize(fl->ev[2][11]);
  for (int k = 0; k < 11; ++k) {
    ms[k] = 0.f;
    for (int l = 0; l < 3 && e == cudaSuccess; ++l) {
      float t = 0.f;
      e = cudaEventElapsedTime(&t, fl->ev[l][k], fl->ev[l][k + 1]);
      ms[k] += t;
    }
  }
  ms[11] = ms[12] = 0.f;
  if (e == cudaSuccess && fl->have_struct) {
    e = cudaEventSynchronize(fl->evs[2]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms[11], fl->evs[0], fl->evs[1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms[12], fl->evs[1], fl->evs[2]);
  }
  if (e != cudaSuccess)
    return flow_err(IBM_ERR_CUDA, std::string("ibm_flow_get_phase_times: ") + cudaGetErrorString(e));
  return IBM_OK;
}
