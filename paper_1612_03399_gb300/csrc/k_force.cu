// Internal forces of the interaction potentials (Sec. 2.3, Eqs.
// elaspot..areapot) and the node update (Sec. 2.3; Sec. 5 step 4).
//
// One block per patch (a contiguous range of a topology's vertices).  The
// block stages the positions of its own and halo vertices in shared memory,
// evaluates every element touching an own vertex exactly once into
// shared-memory contribution slots (4 per edge: a, b and the wings c, d; 3 per
// face), and each own vertex then sums its slots through a CSR list fixed at
// build time.  The summation order never changes, so F_int is bitwise
// deterministic; nothing is written to global memory but the result.
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
#include <cuda_runtime.h>

#include "force_elems.cuh"
#include "ibm_internal.cuh"

namespace ibm {
namespace {

struct Smem {
  float *px, *py, *pz, *cx, *cy, *cz;
  __device__ Vec<float> pos(int i) const { return {px[i], py[i], pz[i]}; }
  __device__ void put(int s, const Vec<float>& f) const {
    cx[s] = f.x;
    cy[s] = f.y;
    cz[s] = f.z;
  }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// MODE 0: F_int only; 1: F_int + F_ext^v and the node update; 2: the
// acceleration (F_int + F_ext^v)/m, zero on clamped nodes, into Fint
template <int MODE>
__global__ void __launch_bounds__(kForceThreads) force_kernel(
    DeviceTables T, StepConsts sc, int32_t V, int32_t F, const float* __restrict__ x,
    const float* __restrict__ v, const float* __restrict__ Fext, float* __restrict__ Fint,
    float* __restrict__ x_out, float* __restrict__ v_out, double* __restrict__ energy) {
  extern __shared__ float sm[];
  const int2 wk = T.work[blockIdx.x];
  const BodyDev B = T.body[wk.x];
  const TopoDev topo = T.topo[B.topo];
  const PatchHdr P = T.patch[topo.patch_off + wk.y];
  Smem S;
  S.px = sm;
  S.py = S.px + P.n_loc;
  S.pz = S.py + P.n_loc;
  S.cx = S.pz + P.n_loc;
  S.cy = S.cx + P.n_slot;
  S.cz = S.cy + P.n_slot;

  for (int i = threadIdx.x; i < P.n_loc; i += blockDim.x) {
    const int gv = B.v_off + __ldg(T.loc_vert + P.loc_off + i);
    S.px[i] = __ldg(x + gv);
    S.py[i] = __ldg(x + V + gv);
    S.pz[i] = __ldg(x + 2 * V + gv);
  }
  const bool want_e = energy != nullptr;
  double eS = 0.0, eB = 0.0, eA = 0.0;
  __syncthreads();

  // edges: spring + bending
  for (int k = threadIdx.x; k < P.n_edge; k += blockDim.x) {
    const PEdge r = T.pedge[P.edge_off + k];
    const int ge = B.e_off + (r.eid & 0x7fffffff);
    const bool hinge = r.l[3] != kNone;
    const Vec<float> pa = S.pos(r.l[0]), pb = S.pos(r.l[1]);
    const Vec<float> pc = hinge ? S.pos(r.l[2]) : pa, pd = hinge ? S.pos(r.l[3]) : pb;
    const float2 cs0 = hinge ? __ldg(T.cs0 + ge) : make_float2(1.f, 0.f);
    Vec<float> fa, fb, fc, fd, us[2], ub[4];
    float es, eb;
    // per-edge constants (van Gelder springs, materials) where the body has them
    const float ks = B.varied ? B.ks * __ldg(T.kse + ge) : B.ks;
    const float kb = B.varied ? B.kb * __ldg(T.kbe + ge) : B.kb;
    edge_forces(pa, pb, pc, pd, hinge, __ldg(T.l0 + ge), cs0.x, cs0.y, ks, kb, fa, fb, fc, fd, us,
                ub, es, eb);
    if (want_e && (r.eid < 0)) {
      eS += (double)es;
      eB += (double)eb;
    }
    // slot layout [role][element]: consecutive threads hit consecutive banks
    S.put(k, fa);
    S.put(P.n_edge + k, fb);
    S.put(2 * P.n_edge + k, fc);
    S.put(3 * P.n_edge + k, fd);
  }
  // Everything above reads only static tables and positions written two
  // launches back; the marker kernel launched just before (it lets this grid
  // start once all its blocks run) produces the body sums and F_ext, so the
  // face part waits for it to complete (a no-op without that launch mode).
  asm volatile("griddepcontrol.wait;" ::: "memory");
  // per-body global-term coefficients from the marker kernel's exact
  // fixed-point area / volume sums
  const float2 cf = body_coef(B, __ldg(T.qsum + 2 * wk.x), __ldg(T.qsum + 2 * wk.x + 1));
  const float cA = cf.x, cV = cf.y;
  // faces: local area, global area, volume
  const int fbase = 4 * P.n_edge;
  for (int k = threadIdx.x; k < P.n_face; k += blockDim.x) {
    const PFace r = T.pface[P.face_off + k];
    Vec<float> f[3], gA[3], gV[3], ua[3];
    float ea;
    const float ka = B.varied ? B.ka * __ldg(T.kaf + B.f_off + r.fid) : B.ka;
    face_forces(S.pos(r.l[0]), S.pos(r.l[1]), S.pos(r.l[2]), __ldg(T.A0f + B.f_off + r.fid), ka,
                cA, cV, f, gA, gV, ua, ea);
    if (MODE != 0) {
      // F_ext^v = sum over the vertex's faces of F_ext / 3: each face adds a
      // third of its load to its corner slots, gathered with the forces
      const int gf = B.f_off + r.fid;
      const float third = 1.f / 3.f;
      const Vec<float> fe = {__ldg(Fext + gf) * third, __ldg(Fext + F + gf) * third,
                             __ldg(Fext + 2 * F + gf) * third};
#pragma unroll
      for (int c = 0; c < 3; ++c) f[c] = vadd(f[c], fe);
    }
    S.put(fbase + k, f[0]);
    S.put(fbase + P.n_face + k, f[1]);
    S.put(fbase + 2 * P.n_face + k, f[2]);
    if (want_e && r.owned) eA += (double)ea;
  }
  __syncthreads();

  // own vertices: fixed-order gather of the slots
  for (int i = threadIdx.x; i < P.n_own; i += blockDim.x) {
    const int s0 = __ldg(T.csr_ptr + P.csr_off + i), s1 = __ldg(T.csr_ptr + P.csr_off + i + 1);
    float fx = 0.f, fy = 0.f, fz = 0.f;
    for (int k = s0; k < s1; ++k) {
      const int s = T.csr_slot[P.slot_off + k];
      fx += S.cx[s];
      fy += S.cy[s];
      fz += S.cz[s];
    }
    const int lv = P.own0 + i;
    const int gv = B.v_off + lv;
    if (MODE == 0) {
      Fint[gv] = fx;
      Fint[V + gv] = fy;
      Fint[2 * V + gv] = fz;
    } else if (MODE == 2) {
      const bool cl = T.clamp[gv] != 0;
      Fint[gv] = cl ? 0.f : fx * B.inv_mass;
      Fint[V + gv] = cl ? 0.f : fy * B.inv_mass;
      Fint[2 * V + gv] = cl ? 0.f : fz * B.inv_mass;
    } else {
      // the gathered slots hold F_int + F_ext^v
      const float ax = fx * B.inv_mass, ay = fy * B.inv_mass, az = fz * B.inv_mass;
      const float x0 = S.px[i], y0 = S.py[i], z0 = S.pz[i];
      float vx = __ldg(v + gv), vy = __ldg(v + V + gv), vz = __ldg(v + 2 * V + gv);
      float nx, ny, nz;
      if (sc.forward_euler) {
        nx = x0 + sc.dt * vx; ny = y0 + sc.dt * vy; nz = z0 + sc.dt * vz;
        vx += sc.dt * ax; vy += sc.dt * ay; vz += sc.dt * az;
      } else {
        vx += sc.dt * ax; vy += sc.dt * ay; vz += sc.dt * az;
        nx = x0 + sc.dt * vx; ny = y0 + sc.dt * vy; nz = z0 + sc.dt * vz;
      }
      if (T.clamp[gv]) {
        nx = x0; ny = y0; nz = z0;
        vx = vy = vz = 0.f;
      }
      x_out[gv] = nx; x_out[V + gv] = ny; x_out[2 * V + gv] = nz;
      v_out[gv] = vx; v_out[V + gv] = vy; v_out[2 * V + gv] = vz;
    }
  }

  if (want_e) {
    __shared__ double red[3][kForceThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    eS = warp_sum(eS);
    eB = warp_sum(eB);
    eA = warp_sum(eA);
    if (lane == 0) {
      red[0][wid] = eS;
      red[1][wid] = eB;
      red[2][wid] = eA;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double a = 0.0, b = 0.0, c = 0.0;
      for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
        a += red[0][k];
        b += red[1][k];
        c += red[2][k];
      }
      atomicAdd(energy + 5 * wk.x + 0, a);
      atomicAdd(energy + 5 * wk.x + 1, b);
      atomicAdd(energy + 5 * wk.x + 2, c);
      if (wk.y == 0) {
        const double Ab = T.meas[2 * wk.x], Vb = T.meas[2 * wk.x + 1];
        energy[5 * wk.x + 3] = 0.5 * B.kA * (Ab - B.A0) * (Ab - B.A0) / B.A0;
        energy[5 * wk.x + 4] = B.closed ? 0.5 * B.kv * (Vb - B.V0) * (Vb - B.V0) / B.V0 : 0.0;
      }
    }
  }
}

// node update with a given F_int (the stand-alone advance entry point)
__global__ void __launch_bounds__(kForceThreads) advance_kernel(
    DeviceTables T, StepConsts sc, int32_t V, int32_t F, const float* __restrict__ x,
    const float* __restrict__ v, const float* __restrict__ Fint, const float* __restrict__ Fext,
    float* __restrict__ x_out, float* __restrict__ v_out) {
  const int2 wk = T.work[blockIdx.x];
  const BodyDev B = T.body[wk.x];
  const TopoDev topo = T.topo[B.topo];
  const PatchHdr P = T.patch[topo.patch_off + wk.y];
  for (int i = threadIdx.x; i < P.n_own; i += blockDim.x) {
    const int lv = P.own0 + i;
    const int gv = B.v_off + lv;
    const int* vp = T.v2f_ptr + topo.v2f_ptr_off;
    const int q0 = __ldg(vp + lv), q1 = __ldg(vp + lv + 1);
    float ex = 0.f, ey = 0.f, ez = 0.f;
    for (int q = q0; q < q1; ++q) {
      const int gf = B.f_off + __ldg(T.v2f_idx + topo.v2f_idx_off + q);
      ex += __ldg(Fext + gf);
      ey += __ldg(Fext + F + gf);
      ez += __ldg(Fext + 2 * F + gf);
    }
    const float third = 1.f / 3.f;
    const float ax = (__ldg(Fint + gv) + ex * third) * B.inv_mass;
    const float ay = (__ldg(Fint + V + gv) + ey * third) * B.inv_mass;
    const float az = (__ldg(Fint + 2 * V + gv) + ez * third) * B.inv_mass;
    const float x0 = __ldg(x + gv), y0 = __ldg(x + V + gv), z0 = __ldg(x + 2 * V + gv);
    float vx = __ldg(v + gv), vy = __ldg(v + V + gv), vz = __ldg(v + 2 * V + gv);
    float nx, ny, nz;
    if (sc.forward_euler) {
      nx = x0 + sc.dt * vx; ny = y0 + sc.dt * vy; nz = z0 + sc.dt * vz;
      vx += sc.dt * ax; vy += sc.dt * ay; vz += sc.dt * az;
    } else {
      vx += sc.dt * ax; vy += sc.dt * ay; vz += sc.dt * az;
      nx = x0 + sc.dt * vx; ny = y0 + sc.dt * vy; nz = z0 + sc.dt * vz;
    }
    if (T.clamp[gv]) {
      nx = x0; ny = y0; nz = z0;
      vx = vy = vz = 0.f;
    }
    x_out[gv] = nx; x_out[V + gv] = ny; x_out[2 * V + gv] = nz;
    v_out[gv] = vx; v_out[V + gv] = vy; v_out[2 * V + gv] = vz;
  }
}

}  // namespace

// Force kernels are launched with programmatic stream serialisation: they
// may start while the preceding marker kernel's last blocks still run (the
// marker kernel allows it from the start of every block) and wait for its
// completion before the face part; after any other preceding work they start
// as usual, when it has completed.
template <int MODE>
cudaError_t launch_force_mode(ibm_ctx* c, const float* x, const float* v, const float* Fext,
                              float* Fint, float* x_out, float* v_out, double* energy) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)c->n_work);
  cfg.blockDim = dim3(kForceThreads);
  cfg.dynamicSmemBytes = c->force_smem;
  cfg.stream = c->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, force_kernel<MODE>, c->d, c->sc, (int32_t)c->V, (int32_t)c->F,
                            x, v, Fext, Fint, x_out, v_out, energy);
}

cudaError_t launch_force(ibm_ctx* c, const float* x, const float* v, const float* Fext,
                         float* Fint, float* x_out, float* v_out, double* energy, bool advance) {
  if (c->n_work == 0) return cudaSuccess;
  return advance ? launch_force_mode<1>(c, x, v, Fext, Fint, x_out, v_out, energy)
                 : launch_force_mode<0>(c, x, v, Fext, Fint, x_out, v_out, energy);
}

cudaError_t launch_accel(ibm_ctx* c, const float* x, const float* Fext, float* a) {
  if (c->n_work == 0) return cudaSuccess;
  return launch_force_mode<2>(c, x, nullptr, Fext, a, nullptr, nullptr, nullptr);
}

cudaError_t launch_advance(ibm_ctx* c, const float* x, const float* v, const float* Fint,
                           const float* Fext, float* x_out, float* v_out) {
  if (c->n_work == 0) return cudaSuccess;
  advance_kernel<<<c->n_work, kForceThreads, 0, c->stream>>>(c->d, c->sc, (int32_t)c->V,
                                                              (int32_t)c->F, x, v, Fint, Fext,
                                                              x_out, v_out);
  return cudaGetLastError();
}

cudaError_t set_force_smem_limit(size_t bytes) {
  cudaError_t e = cudaFuncSetAttribute(force_kernel<1>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(force_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(force_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)bytes);
}

}  // namespace ibm
