// Internal forces of the interaction potentials (Sec. 2.3, Eqs.
// elaspot..areapot) and the node update (Sec. 2.3; Sec. 5 step 4).
//
// One block per patch (a contiguous range of a topology's vertices).  The
// block stages the positions of its own and halo vertices in shared memory,
// evaluates every element touching an own vertex exactly once into
// shared-memory contribution slots, and each own vertex then sums its slots,
// which are contiguous and in an order fixed at build time.  The summation
// order never changes, so F_int is bitwise deterministic; nothing is written
// to global memory but the result.
//
// The patch's element records (with the slot each role writes) and its rest
// data arrive in shared memory with two bulk copies completing on an
// mbarrier, issued first; the position gather runs meanwhile.  After that the
// element loops read shared memory only, so a block waits on global memory
// about three times (positions, the marker kernel's traction, the velocities),
// not once per element.
//
#include <cuda_runtime.h>

#include "bulk_copy.cuh"
#include "force_elems.cuh"
#include "ibm_internal.cuh"

namespace ibm {
namespace {

struct Smem {
  float *px, *py, *pz, *cx, *cy, *cz;
  __device__ Vec<float> pos(int i) const { return {px[i], py[i], pz[i]}; }
  __device__ void put(int s, const Vec<float>& f) const {
    if (s == kNone) return;
    cx[s] = f.x;
    cy[s] = f.y;
    cz[s] = f.z;
  }
  __device__ void add(int s, const Vec<float>& f) const {
    if (s == kNone) return;
    cx[s] += f.x;
    cy[s] += f.y;
    cz[s] += f.z;
  }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}


// Host mirror of x', v' (one block, after its own vertices' writes): count
// this block's entries into the chunks of the flat [3][V] arrays they fall in;
// the block whose entries complete a chunk copies the whole chunk, written by
// whichever blocks, into host memory with contiguous (vector) stores.  Each
// block fences its writes before it counts, and the copying block reads
// through L2, so it sees every block's writes to the chunk.  No block waits.
__device__ __noinline__ void mirror_chunks(Mirror m, const float* x_out, const float* v_out,
                                           int32_t V, int gv0, int n_own) {
  // a run of at most 2048 own vertices (the patch-size limit, which is
  // kMirrorChunk) meets at most two chunks per component
  __shared__ int s_done[6];
  __threadfence();
  __syncthreads();
  const long long total = 3ll * V;
  if (threadIdx.x < 6) {
    // thread 2 d + j: component d, the j-th chunk its run of own vertices meets
    const int d = threadIdx.x >> 1, j = threadIdx.x & 1;
    const long long f0 = (long long)d * V + gv0, f1 = f0 + n_own;   // [f0, f1)
    const long long k = f0 / kMirrorChunk + j;
    int done = -1;
    if (n_own > 0 && k * kMirrorChunk < f1) {
      const long long lo = max(f0, k * kMirrorChunk), hi = min(f1, (k + 1) * kMirrorChunk);
      const int n = (int)(hi - lo);
      const int len = (int)min((long long)kMirrorChunk, total - k * kMirrorChunk);
      if (atomicAdd(m.count + k, n) + n == len) done = (int)k;
    }
    s_done[threadIdx.x] = done;
  }
  __syncthreads();
  for (int t = 0; t < 6; ++t) {
    const int k = s_done[t];
    if (k < 0) continue;   // uniform over the block
    __threadfence();
    const long long b0 = (long long)k * kMirrorChunk;
    const int len = (int)min((long long)kMirrorChunk, total - b0);
    if (m.vec && (len & 3) == 0) {
      const float4* sx = reinterpret_cast<const float4*>(x_out + b0);
      const float4* sv = reinterpret_cast<const float4*>(v_out + b0);
      float4* dx = reinterpret_cast<float4*>(m.hx + b0);
      float4* dv = reinterpret_cast<float4*>(m.hv + b0);
      for (int q = threadIdx.x; q < len / 4; q += blockDim.x) {
        dx[q] = __ldcg(sx + q);
        dv[q] = __ldcg(sv + q);
      }
    } else {
      for (int q = threadIdx.x; q < len; q += blockDim.x) {
        m.hx[b0 + q] = __ldcg(x_out + b0 + q);
        m.hv[b0 + q] = __ldcg(v_out + b0 + q);
      }
    }
  }
}

// MODE 0: F_int only; 1: F_int + F_ext^v and the node update; 2: the
// acceleration (F_int + F_ext^v)/m, zero on clamped nodes, into Fint
template <int MODE>
__global__ void __launch_bounds__(kForceThreads) force_kernel(
    DeviceTables T, StepConsts sc, int32_t V, int32_t F, const float* __restrict__ x,
    const float* __restrict__ v, const float* __restrict__ Fext, float* __restrict__ Fint,
    float* __restrict__ x_out, float* __restrict__ v_out, double* __restrict__ energy,
    Mirror mirror) {
  extern __shared__ __align__(16) float sm[];
  __shared__ __align__(8) unsigned long long bar;
  const int2 wk = T.work[blockIdx.x];
  const BodyDev B = T.body[wk.x];
  const TopoDev topo = T.topo[B.topo];
  const PatchHdr P = T.patch[topo.patch_off + wk.y];
  const FPatch Q = T.fpatch[topo.patch_off + wk.y];
  const int pe = pad4(P.n_edge), pf = pad4(P.n_face);
  const int rest_words = frest_words(P.n_edge, P.n_face, B.varied != 0);
  const uint4* rec = reinterpret_cast<const uint4*>(sm);                   // edges
  const uint2* frec = reinterpret_cast<const uint2*>(sm + 4 * P.n_edge);   // faces
  const uint16_t* ptr = reinterpret_cast<const uint16_t*>(sm + 4 * P.n_edge + 2 * P.n_face);
  const float* rest = sm + Q.blob_words;
  Smem S;
  S.px = sm + Q.blob_words + rest_words;
  S.py = S.px + pad4(P.n_loc);
  S.pz = S.py + pad4(P.n_loc);
  S.cx = S.pz + pad4(P.n_loc);
  S.cy = S.cx + pad4(Q.n_slot);
  S.cz = S.cy + pad4(Q.n_slot);

  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    const unsigned nb = 4u * (unsigned)Q.blob_words, nr = 4u * (unsigned)rest_words;
    mbar_arrive_tx(&bar, nb + nr + (unsigned)sc.starve_tx);
    if (nb) bulk_load(sm, T.fblob + Q.blob_off, nb, &bar);
    if (nr) bulk_load(sm + Q.blob_words, T.frest + T.wrest[blockIdx.x], nr, &bar);
  }
  // meanwhile: positions of the own and halo vertices, two per thread in flight
  for (int i = threadIdx.x; i < P.n_loc; i += 2 * blockDim.x) {
    const int j = i + blockDim.x;
    const int gi = B.v_off + __ldg(T.loc_vert + P.loc_off + i);
    const int gj = j < P.n_loc ? B.v_off + __ldg(T.loc_vert + P.loc_off + j) : gi;
    const float xi = __ldg(x + gi), yi = __ldg(x + V + gi), zi = __ldg(x + 2 * V + gi);
    const float xj = __ldg(x + gj), yj = __ldg(x + V + gj), zj = __ldg(x + 2 * V + gj);
    S.px[i] = xi;
    S.py[i] = yi;
    S.pz[i] = zi;
    if (j < P.n_loc) {
      S.px[j] = xj;
      S.py[j] = yj;
      S.pz[j] = zj;
    }
  }
  // and the velocity and clamp flag of the thread's first own vertex
  float pv[3] = {0.f, 0.f, 0.f};
  bool pcl = false;
  if (MODE == 1 && (int)threadIdx.x < P.n_own) {
    const int gv = B.v_off + P.own0 + threadIdx.x;
    pv[0] = __ldg(v + gv);
    pv[1] = __ldg(v + V + gv);
    pv[2] = __ldg(v + 2 * V + gv);
    pcl = T.clamp[gv] != 0;
  }
  const bool want_e = energy != nullptr;
  double eS = 0.0, eB = 0.0, eA = 0.0;
  __syncthreads();   // positions staged, barrier initialised
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

  // edges: spring + bending, from shared memory only
  for (int k = threadIdx.x; k < P.n_edge; k += blockDim.x) {
    const uint4 r = rec[k];
    const int la = r.x & 0xFFFF, lb = r.x >> 16, lc = r.y & 0xFFFF, ld = r.y >> 16;
    const bool hinge = ld != kNone;
    const Vec<float> pa = S.pos(la), pb = S.pos(lb);
    const Vec<float> pc = hinge ? S.pos(lc) : pa, pd = hinge ? S.pos(ld) : pb;
    const float c0 = hinge ? rest[pe + k] : 1.f, s0 = hinge ? rest[2 * pe + k] : 0.f;
    Vec<float> fa, fb, fc, fd, us[2], ub[4];
    float es, eb;
    // per-edge constants (van Gelder springs, materials) where the body has them
    const float ks = B.varied ? B.ks * rest[3 * pe + pf + k] : B.ks;
    const float kb = B.varied ? B.kb * rest[4 * pe + pf + k] : B.kb;
    edge_forces(pa, pb, pc, pd, hinge, rest[k], c0, s0, ks, kb, fa, fb, fc, fd, us, ub, es, eb);
    if (want_e && (r.z & 0xFFFF) != kNone) {   // the patch of vertex a owns the edge
      eS += (double)es;
      eB += (double)eb;
    }
    S.put(r.z & 0xFFFF, fa);
    S.put(r.z >> 16, fb);
    S.put(r.w & 0xFFFF, fc);
    S.put(r.w >> 16, fd);
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
  __syncthreads();   // every edge slot written
  // faces: local area, global area, volume, added to the slots of the edge
  // each face is attached to (an edge per face: no two threads touch the same
  // slot); two faces per thread with their tractions in flight
  const float third = 1.f / 3.f;
  for (int k0 = threadIdx.x; k0 < P.n_face; k0 += 2 * blockDim.x) {
    const int k1 = k0 + blockDim.x;
    const bool two = k1 < P.n_face;
    const uint2 r0 = frec[k0];
    const uint2 r1 = two ? frec[k1] : r0;
    Vec<float> fe0 = {0.f, 0.f, 0.f}, fe1 = {0.f, 0.f, 0.f};
    if (MODE != 0) {
      // F_ext^v = sum over the vertex's faces of F_ext / 3: each face adds a
      // third of its load to its corners, gathered with the forces
      const int g0 = B.f_off + (int)r0.y, g1 = B.f_off + (int)r1.y;
      fe0 = {__ldg(Fext + g0), __ldg(Fext + F + g0), __ldg(Fext + 2 * F + g0)};
      fe1 = {__ldg(Fext + g1), __ldg(Fext + F + g1), __ldg(Fext + 2 * F + g1)};
    }
#pragma unroll 1
    for (int h = 0; h < (two ? 2 : 1); ++h) {
      const uint2 fr = h ? r1 : r0;
      const int k = h ? k1 : k0;
      const uint4 r = rec[fr.x & 0x3FFFFFFFu];
      const bool right = (fr.x >> 30) & 1u;
      const int la = r.x & 0xFFFF, lb = r.x >> 16;
      const int v0 = right ? lb : la, v1 = right ? la : lb;
      const int v2 = right ? (int)(r.y >> 16) : (int)(r.y & 0xFFFF);
      const int d0 = right ? (int)(r.z >> 16) : (int)(r.z & 0xFFFF);
      const int d1 = right ? (int)(r.z & 0xFFFF) : (int)(r.z >> 16);
      const int d2 = right ? (int)(r.w >> 16) : (int)(r.w & 0xFFFF);
      Vec<float> f[3], gA[3], gV[3], ua[3];
      float ea;
      const float ka = B.varied ? B.ka * rest[5 * pe + pf + k] : B.ka;
      face_forces(S.pos(v0), S.pos(v1), S.pos(v2), rest[3 * pe + k], ka, cA, cV, f, gA, gV, ua,
                  ea);
      if (MODE != 0) {
        const Vec<float> fe = vscale(h ? fe1 : fe0, third);
#pragma unroll
        for (int c = 0; c < 3; ++c) f[c] = vadd(f[c], fe);
      }
      S.add(d0, f[0]);
      S.add(d1, f[1]);
      S.add(d2, f[2]);
      if (want_e && (fr.x >> 31)) eA += (double)ea;
    }
  }
  __syncthreads();

  // own vertices: fixed-order sum of their contiguous slots
  for (int i = threadIdx.x; i < P.n_own; i += blockDim.x) {
    const int s0 = ptr[i], s1 = ptr[i + 1];
    float fx = 0.f, fy = 0.f, fz = 0.f;
    for (int s = s0; s < s1; ++s) {
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
      const bool first = i == (int)threadIdx.x;
      float vx = first ? pv[0] : __ldg(v + gv), vy = first ? pv[1] : __ldg(v + V + gv),
            vz = first ? pv[2] : __ldg(v + 2 * V + gv);
      const bool clamped = first ? pcl : T.clamp[gv] != 0;
      float nx, ny, nz;
      if (sc.forward_euler) {
        nx = x0 + sc.dt * vx; ny = y0 + sc.dt * vy; nz = z0 + sc.dt * vz;
        vx += sc.dt * ax; vy += sc.dt * ay; vz += sc.dt * az;
      } else {
        vx += sc.dt * ax; vy += sc.dt * ay; vz += sc.dt * az;
        nx = x0 + sc.dt * vx; ny = y0 + sc.dt * vy; nz = z0 + sc.dt * vz;
      }
      if (clamped) {
        nx = x0; ny = y0; nz = z0;
        vx = vy = vz = 0.f;
      }
      x_out[gv] = nx; x_out[V + gv] = ny; x_out[2 * V + gv] = nz;
      v_out[gv] = vx; v_out[V + gv] = vy; v_out[2 * V + gv] = vz;
    }
  }
  if (MODE == 1 && mirror.hx) mirror_chunks(mirror, x_out, v_out, V, B.v_off + P.own0, P.n_own);

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
                              float* Fint, float* x_out, float* v_out, double* energy,
                              const Mirror& mirror = Mirror()) {
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
                            x, v, Fext, Fint, x_out, v_out, energy, mirror);
}

cudaError_t launch_force(ibm_ctx* c, const float* x, const float* v, const float* Fext,
                         float* Fint, float* x_out, float* v_out, double* energy, bool advance,
                         const Mirror* mirror) {
  if (c->n_work == 0) return cudaSuccess;
  return advance ? launch_force_mode<1>(c, x, v, Fext, Fint, x_out, v_out, energy,
                                        mirror ? *mirror : Mirror())
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
