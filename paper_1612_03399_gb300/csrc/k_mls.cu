// Marker kernel: face geometry, per-body area/volume reductions, MLS
// interpolation at the centroid, direct-forcing marker force, probe gradient
// and traction, and spreading (Sec. 2.2, Eqs. mls..mls_cl; Sec. 5 steps 1-3).
//
// One block = one surface patch of ONE body (up to 128 or 256 faces, built by
// recursive coordinate bisection of the rest mesh), one thread per face.
// The block builds a ROW MAP of its grid footprint: for every (y, z) row of
// the nodes its 3x3x3 supports (centroids and probe ends) touch, the x-range
// touched, padded to whole groups of 4 nodes (float4-aligned when the grid
// allows).  The velocity components are staged in shared memory with
// asynchronous copies, two buffers in flight, and interpolated and
// differentiated from there.  The spread then accumulates one force component
// at a time in exact fixed point (32-bit shared atomics on two words, a
// power-of-two scale per block and component) and flushes it with float4
// global atomics; the rows that received a nonzero spread are recorded so the
// next step's clear zeroes exactly those.  A patch whose footprint does not
// fit takes the direct global path (scalar loads and float atomics) and
// records its bounding box.
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

#include "bulk_copy.cuh"
#include "ibm_internal.cuh"
#include "mls_closed_form.cuh"

namespace ibm {
namespace {

// The global-memory path of a marker block whose footprint does not fit its
// shared memory (rare): out of line, so that it does not crowd the
// instruction cache of the staged path it sits beside.
__device__ __noinline__ float value_global(const float* f, Grid g, int c0, int c1, int c2, DirW X,
                                          DirW Y, DirW Z) {
  const int c[3] = {c0, c1, c2};
  return mls_value(f, GlobalRows{g}.at(c), X, Y, Z);
}
__device__ __noinline__ float3 gradient_global(const float* f, Grid g, ProbeW P, float sgn) {
  float gr[3] = {0.f, 0.f, 0.f};
  P.add_gradient(f, GlobalRows{g}, g.invh, sgn, gr);
  return make_float3(gr[0], gr[1], gr[2]);
}
__device__ __noinline__ void spread_global(float* f, Grid g, int c0, int c1, int c2, DirW X,
                                           DirW Y, DirW Z, float coef) {
  const int c[3] = {c0, c1, c2};
  mls_spread(f, GlobalRows{g}.at(c), X, Y, Z, coef);
}


// REC (record mode): instead of spreading, write each marker's spread record
// (centroid in cells, c_l F) and count it under the tiles of the tile-owned
// spread, with the tile's largest |c_l F| per component
template <int MT, bool MEASURE, bool INTERP, bool PROBE, bool SPREAD, bool REC>
__global__ void __launch_bounds__(MT, 512 / MT) marker_kernel(
    DeviceTables T, Grid g, StepConsts sc, int32_t V, int32_t F, const float* __restrict__ x,
    const float* __restrict__ v, const float* __restrict__ u, const float* __restrict__ vv,
    const float* __restrict__ w, const float* __restrict__ pr, const float* __restrict__ accel,
    float* __restrict__ U, float* __restrict__ Fm, const float* __restrict__ Fm_in,
    float* __restrict__ Fext, float* __restrict__ fx, float* __restrict__ fy,
    float* __restrict__ fz, int record, int vec4, TileDev td, int tmode, float phi_bound_all,
    int cache, int* __restrict__ cache_tab, float4* __restrict__ cache_face) {
  constexpr bool FIELD = INTERP || PROBE || SPREAD;
  // the coupled forcing launch (interpolation and spread at the centroids)
  // may save its face geometry and row tables (cache 1) and, in the later
  // substeps of the same step, load them instead of recomputing (cache 2)
  constexpr bool CACHEABLE = !MEASURE && INTERP && !PROBE && SPREAD && !REC;
  const bool load = CACHEABLE && cache == 2;
  const bool save = CACHEABLE && cache == 1;
  constexpr bool VEL = INTERP || PROBE;
  constexpr bool ROWMAP = VEL || (SPREAD && !REC);
  extern __shared__ __align__(16) unsigned char dyn[];
  constexpr int MR = marker_rows(MT), MN = marker_nodes(MT);   // (y, z) rows, staged nodes
  int* s_xmin = reinterpret_cast<int*>(dyn);   // [MR]  then: staged offset - x0
  int* s_xmax = s_xmin + MR;                   // [MR]  then: row length
  int* s_off = s_xmax + MR;                    // [MR + 4] staged row start
  int* s_nzlo = s_off + MR + 4;                // [MR] first / last group of the row
  int* s_nzhi = s_nzlo + MR;                   //   that received a nonzero spread
  int* s_gofs = s_nzhi + MR;                   // [MN/4] global offset of each group
  unsigned short* s_grow = reinterpret_cast<unsigned short*>(s_gofs + MN / 4);  // row ids
  float* bufA = reinterpret_cast<float*>(dyn + marker_row_table_bytes(MT));
  float* bufB = bufA + MN;
  __shared__ int s_lo[3], s_hi[3];
  __shared__ int s_N;
  __shared__ int s_warp[MT / 32];
  __shared__ int s_bmax[3];
  __shared__ __align__(8) unsigned long long s_bar;
  __shared__ unsigned long long s_q[2][MT / 32];   // per-warp fixed-point body sums

  // a force kernel launched after this one may start once every block of
  // this grid runs (it waits for this grid's results before using them)
  asm volatile("griddepcontrol.launch_dependents;");
  const int4 ch = T.chunks[blockIdx.x];  // body, face-list offset, count, chunk index in body
  const BodyDev B = T.body[ch.x];
  const TopoDev topo = T.topo[B.topo];
  const bool active = threadIdx.x < ch.z;
  if (FIELD && threadIdx.x < 3) {
    s_lo[threadIdx.x] = INT_MAX;
    s_hi[threadIdx.x] = INT_MIN;
    s_bmax[threadIdx.x] = 0;
  }
  if (ROWMAP && !load) {
    // every row's x-range and nonzero range start empty; done first, so that
    // the stores overlap the geometry loads (the barriers of the bounding-box
    // reduction make them visible)
    for (int r = threadIdx.x; r < MR; r += blockDim.x) {
      s_xmin[r] = INT_MAX;
      s_xmax[r] = INT_MIN;
      s_nzlo[r] = INT_MAX;
      s_nzhi[r] = INT_MIN;
    }
  }
  float Af = 0.f, Vf = 0.f;
  float nrm[3] = {0.f, 0.f, 0.f}, area = 0.f;
  float tc[3] = {0.f, 0.f, 0.f}, tp[3] = {0.f, 0.f, 0.f}, tm[3] = {0.f, 0.f, 0.f};
  float vb[3] = {0.f, 0.f, 0.f};     // centroid velocity (interpolation) or marker force
  float am[3] = {0.f, 0.f, 0.f};     // marker acceleration
  bool ok = false;
  int gf = 0;
  if (load && active) {
    const float4 c0 = cache_face[2 * ((size_t)blockIdx.x * kMT + threadIdx.x)];
    const float4 c1 = cache_face[2 * ((size_t)blockIdx.x * kMT + threadIdx.x) + 1];
    tc[0] = c0.x; tc[1] = c0.y; tc[2] = c0.z;
    area = c0.w;
    vb[0] = c1.x; vb[1] = c1.y; vb[2] = c1.z;
    ok = c1.w != 0.f;
  }
  if (active && !load) {
    // full patches are stored so that a warp's faces are spread over the patch
    // (its shared atomics of the spread rarely meet on a node) while thread t
    // reads record t
    const int4 mt = __ldg(T.mtri + topo.mface_off + ch.y + threadIdx.x);
    gf = B.f_off + mt.w;
    const int ia = B.v_off + mt.x, ib = B.v_off + mt.y, ic = B.v_off + mt.z;
    float xa[3], xb[3], xc[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      xa[d] = __ldg(x + d * V + ia);
      xb[d] = __ldg(x + d * V + ib);
      xc[d] = __ldg(x + d * V + ic);
    }
    // issued now, used after the row map: the velocity of the centroid
    // (interpolation) or the given marker force (spread only)
    if (INTERP) {
      const float third = 1.f / 3.f;
#pragma unroll
      for (int d = 0; d < 3; ++d)
        vb[d] = (__ldg(v + d * V + ia) + __ldg(v + d * V + ib) + __ldg(v + d * V + ic)) * third;
    } else if (SPREAD) {
#pragma unroll
      for (int d = 0; d < 3; ++d) vb[d] = __ldg(Fm_in + d * F + gf);
    }
    // marker acceleration (pressure correction): mean of the vertices'
    if (PROBE && pr && accel) {
      const float third = 1.f / 3.f;
#pragma unroll
      for (int d = 0; d < 3; ++d)
        am[d] = (__ldg(accel + d * V + ia) + __ldg(accel + d * V + ib) +
                 __ldg(accel + d * V + ic)) * third;
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
        const float c = (xa[d] + xb[d] + xc[d]) * third;
        nrm[d] = N[d] * inv;
        tc[d] = fmaf(c, g.invh[d], B.frac[d]);
        tp[d] = fmaf(c + sc.probe_h * nrm[d], g.invh[d], B.frac[d]);
        tm[d] = fmaf(c - sc.probe_h * nrm[d], g.invh[d], B.frac[d]);
        ok = ok && fabsf(tc[d]) < 4.0e6f && fabsf(tp[d]) < 4.0e6f && fabsf(tm[d]) < 4.0e6f;
      }
      if (!ok) atomicOr(T.err, ERR_NONFINITE);
    }
    if (save) {
      cache_face[2 * ((size_t)blockIdx.x * kMT + threadIdx.x)] = make_float4(tc[0], tc[1], tc[2], area);
      cache_face[2 * ((size_t)blockIdx.x * kMT + threadIdx.x) + 1] =
          make_float4(vb[0], vb[1], vb[2], ok ? 1.f : 0.f);
    }
  }

  // ---- per-body area and volume: exact fixed-point sums -------------------
  // q = rint(value * 2^e) per face (2^e from the rest value), summed per warp
  // and added with 64-bit integer atomics: the body's sum does not depend on
  // the order of the additions
  if (MEASURE) {
    long long qa = 0, qv = 0;
    if (active) {
      const float ya = Af * B.sA, yv = Vf * B.sV;
      if (fabsf(ya) < B.qlim && fabsf(yv) < B.qlim) {
        qa = to_fixed(ya);
        qv = to_fixed(yv);
      } else {
        atomicOr(T.err, ERR_NONFINITE);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      qa += __shfl_xor_sync(0xffffffffu, qa, o);
      qv += __shfl_xor_sync(0xffffffffu, qv, o);
    }
    // added to the body's sums after the wait below (a footprint clear
    // launched before this kernel zeroes them)
    if ((threadIdx.x & 31) == 0) {
      s_q[0][threadIdx.x >> 5] = (unsigned long long)qa;
      s_q[1][threadIdx.x >> 5] = (unsigned long long)qv;
    }
  }

  const bool mine = FIELD && active && ok;
  const bool two = PROBE && !B.closed;     // open sheet: probes on both sides

  // ---- row map of the block's footprint -----------------------------------
  int ylo = 0, zlo = 0, sy = 0, sz = 0, xlo = 0, sx = 0;
  bool fit = false;
  int N = 0;
  if (ROWMAP && load) {
    // the tables of substep 0 of this coupled step: header, then one bulk
    // copy per row array and one for the group -> row table
    const int* hd = cache_tab + (size_t)blockIdx.x * kCacheWords;
    xlo = hd[0];
    ylo = hd[1];
    zlo = hd[2];
    sx = hd[3];
    sy = hd[4];
    sz = hd[5];
    N = hd[6];
    fit = hd[7] != 0;
    const int nrows = fit ? sy * sz : 0;
    if (threadIdx.x == 0) {
      mbar_init(&s_bar, 1);
      const unsigned rb = 4u * (unsigned)pad4(nrows);
      const unsigned ob = fit ? 4u * (unsigned)pad4(N / 4) : 0u;
      const unsigned gb = fit ? 2u * (unsigned)((N / 4 + 7) & ~7) : 0u;
      mbar_arrive_tx(&s_bar, 3u * rb + ob + gb + (unsigned)sc.starve_tx);
      if (fit) {
        const int* src = hd + 16;
        bulk_load(s_xmin, src, rb, &s_bar);
        bulk_load(s_xmax, src + kMaxRows, rb, &s_bar);
        bulk_load(s_off, src + 2 * kMaxRows, rb, &s_bar);
        bulk_load(s_gofs, src + 3 * kMaxRows, ob, &s_bar);
        bulk_load(s_grow, src + 3 * kMaxRows + kMaxNodes / 4, gb, &s_bar);
      }
      s_off[MR] = N;
    }
    for (int r = threadIdx.x; r < nrows; r += blockDim.x) {
      s_nzlo[r] = INT_MAX;
      s_nzhi[r] = INT_MIN;
    }
    __syncthreads();   // barrier initialised
    if (!__syncthreads_and(mbar_wait(&s_bar, kCopyWaitClocks))) {
      // the copies did not land: flag it, give them one more bounded wait
      // (they write this block's shared memory) and leave
      if (threadIdx.x == 0) {
        atomicOr(T.err, ERR_TIMEOUT);
        mbar_wait(&s_bar, kCopyWaitClocks);
      }
      __syncthreads();
      return;
    }
    if (!fit && threadIdx.x == 0) atomicAdd(T.stats, 1);
  } else if (ROWMAP) {
    int mlo[3] = {INT_MAX, INT_MAX, INT_MAX}, mhi[3] = {INT_MIN, INT_MIN, INT_MIN};
    if (mine) {
#pragma unroll
      for (int l = 0; l < 3; ++l) {
        if ((l == 1 && !PROBE) || (l == 2 && !two)) continue;
        const float(&t)[3] = l == 0 ? tc : (l == 1 ? tp : tm);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const int f0 = B.G[d] + (int)floorf(t[d]);
          mlo[d] = min(mlo[d], f0 - 2);    // generous: every support lies in f0-1 .. f0+2
          mhi[d] = max(mhi[d], f0 + 3);
        }
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
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        atomicMin(&s_lo[d], mlo[d]);
        atomicMax(&s_hi[d], mhi[d]);
      }
    }
    __syncthreads();
    xlo = s_lo[0];
    ylo = s_lo[1];
    zlo = s_lo[2];
    sx = s_hi[0] >= s_lo[0] ? s_hi[0] - s_lo[0] + 1 : 0;
    sy = s_hi[1] >= s_lo[1] ? s_hi[1] - s_lo[1] + 1 : 0;
    sz = s_hi[2] >= s_lo[2] ? s_hi[2] - s_lo[2] + 1 : 0;
    const long long nrows = (long long)sy * sz;
    const bool rows_ok = nrows > 0 && nrows <= MR && sx <= 30000;
    if (rows_ok) {
      if (mine) {
        // every component's support at a point with f = floor(tau) lies in
        // the 4x4x4 window f - 1 .. f + 2 (the nearest-node choice is exact
        // for |tau| < 2^22, which the position check guarantees)
#pragma unroll 1
        for (int l = 0; l < 3; ++l) {
          if ((l == 1 && !PROBE) || (l == 2 && !two)) continue;
          const float(&t)[3] = l == 0 ? tc : (l == 1 ? tp : tm);
          const int fx0 = B.G[0] + (int)floorf(t[0]) - 1;
          const int r0 = (B.G[1] + (int)floorf(t[1]) - 1 - ylo) +
                         sy * (B.G[2] + (int)floorf(t[2]) - 1 - zlo);
#pragma unroll
          for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              atomicMin(&s_xmin[r0 + j + sy * k], fx0);
              atomicMax(&s_xmax[r0 + j + sy * k], fx0 + 3);
            }
        }
      }
      __syncthreads();
      // row lengths in whole groups of 4 nodes (aligned to float4 in global
      // memory when the grid allows vector access) and their exclusive scan;
      // thread t owns rows 4t .. 4t + 3 here
      int len[4], st[4], run = 0;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = 4 * threadIdx.x + q;
        int L = 0, a = 0;
        if (r < (int)nrows && s_xmin[r] <= s_xmax[r]) {
          a = s_xmin[r];
          int b = s_xmax[r] + 1;
          if (vec4) {
            a &= ~3;             // floor to a multiple of 4 (two's complement)
            b = (b + 3) & ~3;
          } else {
            b = a + ((b - a + 3) & ~3);
          }
          L = b - a;
        }
        len[q] = L;
        st[q] = a;
        run += L;
      }
      // block exclusive scan of run
      int incl = run;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if ((threadIdx.x & 31) >= o) incl += t;
      }
      if ((threadIdx.x & 31) == 31) s_warp[threadIdx.x >> 5] = incl;
      __syncthreads();
      int base = 0;
      for (int k = 0; k < (int)(threadIdx.x >> 5); ++k) base += s_warp[k];
      int pos = base + incl - run;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = 4 * threadIdx.x + q;
        if (r < MR) {
          s_off[r] = pos;
          s_xmax[r] = len[q];
          s_xmin[r] = st[q];
        }
        pos += len[q];
      }
      if (threadIdx.x == blockDim.x - 1) {
        s_N = pos;
        s_off[MR] = pos;
      }
      __syncthreads();
      N = s_N;
      fit = N <= MN;
      // per row, strided over the whole block: group -> row ids, global row
      // offset, wrapped first x and staged offset - x0 (row r is (y, z) =
      // (r % sy, r / sy), followed incrementally)
      {
        int yy = (int)threadIdx.x % sy, zz = (int)threadIdx.x / sy;
        const int dy = (int)blockDim.x % sy, dz = (int)blockDim.x / sy;
        for (int r = threadIdx.x; r < (int)nrows; r += blockDim.x) {
          const int L = s_xmax[r];
          if (L > 0) {
            const int p0 = s_off[r], a = s_xmin[r];
            const int base = (wrap(zlo + zz, g.n[2]) * g.n[1] + wrap(ylo + yy, g.n[1])) * g.n[0];
            const int x0w = wrap(a, g.n[0]);
            // groups past MN / 4 only occur when the block does not fit
            const int q1 = min((p0 + L) / 4, MN / 4);
            for (int k = p0 / 4; k < q1; ++k) {
              s_grow[k] = (unsigned short)r;
              s_gofs[k] = base + wrap_pos(x0w + 4 * (k - p0 / 4), g.n[0]);
            }
            s_xmin[r] = p0 - a;
          }
          yy += dy;
          zz += dz;
          if (yy >= sy) {
            yy -= sy;
            ++zz;
          }
        }
      }
    }
    if (!fit && threadIdx.x == 0) atomicAdd(T.stats, 1);
    __syncthreads();
    if (save) {
      int* hd = cache_tab + (size_t)blockIdx.x * kCacheWords;
      if (threadIdx.x == 0) {
        hd[0] = xlo;
        hd[1] = ylo;
        hd[2] = zlo;
        hd[3] = sx;
        hd[4] = sy;
        hd[5] = sz;
        hd[6] = N;
        hd[7] = fit ? 1 : 0;
      }
      if (fit) {
        int* dst = hd + 16;
        for (int r = threadIdx.x; r < sy * sz; r += blockDim.x) {
          dst[r] = s_xmin[r];
          dst[kMaxRows + r] = s_xmax[r];
          dst[2 * kMaxRows + r] = s_off[r];
        }
        unsigned short* gg = reinterpret_cast<unsigned short*>(dst + 3 * kMaxRows + kMaxNodes / 4);
        for (int q = threadIdx.x; q < N / 4; q += blockDim.x) {
          dst[3 * kMaxRows + q] = s_gofs[q];
          gg[q] = s_grow[q];
        }
      }
    }
  }
  const RowTable RT{s_gofs, g.n[0], vec4};
  const StagedRows SR{s_xmin, ylo, zlo, sy};
  const int ngroups = fit ? N / 4 : 0;

  // ---- velocity: interpolation at the centroid, gradient at the probes -----
  // The three components are staged in two buffers (u -> A, v -> B, w -> A),
  // the copies of the next component in flight while the current one is used.
  // Traction t = (G + G^T) n: component i yields (G n)_i and adds n_i G_i. to
  // G^T n.
  float Fl[3] = {vb[0], vb[1], vb[2]};   // marker force per component
  if (VEL) {
    float tGn[3] = {0.f, 0.f, 0.f}, tGTn[3] = {0.f, 0.f, 0.f};
    // with a pressure field it is staged as a fourth component (u -> A,
    // v -> B, w -> A, p -> B); the jump P = p+ - p- (open) or p (closed)
    const bool press = PROBE && pr != nullptr;
    float Pj = 0.f;
    if (fit) {
      stage_async(bufA, u, RT, ngroups);
      cp_async_commit();
      stage_async(bufB, vv, RT, ngroups);
      cp_async_commit();
    }
    // the components in a loop, not unrolled: the unrolled kernel measured
    // slower (instruction fetch stalls)
#pragma unroll 1
    for (int comp = 0; comp < (press ? 4 : 3); ++comp) {
      const float* velc = comp == 0 ? u : (comp == 1 ? vv : (comp == 2 ? w : pr));
      const float* buf = (comp & 1) ? bufB : bufA;
      // the centroid's factors first: their arithmetic overlaps the copies
      // still in flight (the probe's as well would not fit in registers)
      DirW CX, CY, CZ;
      int ccC[3];
      if (INTERP && mine && comp < 3) {
        float t3[3];
        locate(tc, comp, B.G, ccC, t3);
        dir_weights(t3[0], sc.kappa, CX);
        dir_weights(t3[1], sc.kappa, CY);
        dir_weights(t3[2], sc.kappa, CZ);
      }
      if (fit) {
        // one later group (the next component) may still be in flight
        if (comp < 2 || (comp == 2 && press)) cp_async_wait<1>(); else cp_async_wait<0>();
        __syncthreads();   // every thread's copies of this component have landed
      }
      if (mine && comp == 3) {
        // probe pressure p* and the correction h (Du/Dt).n, per side with its
        // own normal: P = p*+ + h a.n (closed), p*+ - p*- + 2 h a.n (open)
        const float an = am[0] * nrm[0] + am[1] * nrm[1] + am[2] * nrm[2];
#pragma unroll 1
        for (int l = 0; l < (two ? 2 : 1); ++l) {
          int cc[3];
          float t3[3];
          locate(l == 0 ? tp : tm, 3, B.G, cc, t3);
          DirW X, Y, Z;
          dir_weights(t3[0], sc.kappa, X);
          dir_weights(t3[1], sc.kappa, Y);
          dir_weights(t3[2], sc.kappa, Z);
          const float ps = fit ? mls_value(buf, SR.at(cc), X, Y, Z)
                               : value_global(pr, g, cc[0], cc[1], cc[2], X, Y, Z);
          Pj += (l == 0 ? 1.f : -1.f) * ps + sc.probe_h * an;
        }
      } else if (mine) {
        if (PROBE) {
          // open sheet: (tau+ - tau-) . n+
          float gr[3] = {0.f, 0.f, 0.f};
          ProbeW P0;
          P0.prepare(tp, comp, B.G, sc.kappa);
          if (fit) {
            P0.add_gradient(buf, SR, g.invh, 1.f, gr);
          } else {
            const float3 q = gradient_global(velc, g, P0, 1.f);
            gr[0] += q.x;
            gr[1] += q.y;
            gr[2] += q.z;
          }
          if (two) {
            ProbeW P1;
            P1.prepare(tm, comp, B.G, sc.kappa);
            if (fit) {
              P1.add_gradient(buf, SR, g.invh, -1.f, gr);
            } else {
              const float3 q = gradient_global(velc, g, P1, -1.f);
              gr[0] += q.x;
              gr[1] += q.y;
              gr[2] += q.z;
            }
          }
          const float gn = gr[0] * nrm[0] + gr[1] * nrm[1] + gr[2] * nrm[2];
          const float ni = comp == 0 ? nrm[0] : (comp == 1 ? nrm[1] : nrm[2]);
          if (comp == 0) tGn[0] = gn;
          if (comp == 1) tGn[1] = gn;
          if (comp == 2) tGn[2] = gn;
#pragma unroll
          for (int j = 0; j < 3; ++j) tGTn[j] += ni * gr[j];
        }
        if (INTERP) {
          const float Ul = fit ? mls_value(buf, SR.at(ccC), CX, CY, CZ)
                               : value_global(velc, g, ccC[0], ccC[1], ccC[2], CX, CY, CZ);
          const float Fc = ((comp == 0 ? vb[0] : (comp == 1 ? vb[1] : vb[2])) - Ul) * sc.inv_dt;
          if (comp == 0) Fl[0] = Fc;
          if (comp == 1) Fl[1] = Fc;
          if (comp == 2) Fl[2] = Fc;
          if (U) U[comp * F + gf] = Ul;
          if (Fm) Fm[comp * F + gf] = Fc;
        }
      }
      if (fit && comp == 0) {
        __syncthreads();   // buffer A is free again
        stage_async(bufA, w, RT, ngroups);
        cp_async_commit();
      }
      if (fit && comp == 1 && press) {
        __syncthreads();   // buffer B is free again
        stage_async(bufB, pr, RT, ngroups);
        cp_async_commit();
      }
    }
    if (PROBE && mine) {
      const float s = sc.mu * area;
#pragma unroll
      for (int i = 0; i < 3; ++i) Fext[i * F + gf] = s * (tGn[i] + tGTn[i]) - area * Pj * nrm[i];
    }
  }

  // ---- records of the tile-owned spread ------------------------------------
  if (REC && active) {
    float4 r0 = make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
    float4 r1 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (mine) {
      const float cl = area * sc.cl_scale;
      r0 = make_float4(tc[0], tc[1], tc[2], __int_as_float(ch.x));
      r1 = make_float4(cl * Fl[0], cl * Fl[1], cl * Fl[2], 0.f);
      int tx[3], ty[3], tz[3];
      const int nx_ = tiles_along(B.G[0] + (int)floorf(tc[0]), g.n[0], kTX, tx);
      const int ny_ = tiles_along(B.G[1] + (int)floorf(tc[1]), g.n[1], kTY, ty);
      const int nz_ = tiles_along(B.G[2] + (int)floorf(tc[2]), g.n[2], kTZ, tz);
      const unsigned m0 = __float_as_uint(fabsf(r1.x)), m1 = __float_as_uint(fabsf(r1.y)),
                     m2 = __float_as_uint(fabsf(r1.z));
      // reductions without a returned value: nothing waits on them
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
          for (int c = 0; c < 3; ++c)
            if (a < nz_ && b < ny_ && c < nx_) {
              const int t = (tz[a] * td.nt[1] + ty[b]) * td.nt[0] + tx[c];
              atomicAdd(td.count + t, 1);
              atomicMax(td.tmax + 4 * (size_t)t, m0);
              atomicMax(td.tmax + 4 * (size_t)t + 1, m1);
              atomicMax(td.tmax + 4 * (size_t)t + 2, m2);
            }
    }
    td.rec[2 * (size_t)gf] = r0;
    td.rec[2 * (size_t)gf + 1] = r1;
  }

  // Everything above reads only inputs.  What follows meets the footprint
  // clear of the step, which may be the grid launched just before this one
  // (this kernel may then start while the clear still runs): the body sums
  // it zeroes, the fields and the footprint record.  Wait for that grid to
  // complete (immediate when nothing precedes programmatically).
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (MEASURE && (threadIdx.x & 31) == 0 && (threadIdx.x >> 5) * 32 < ch.z) {
    atomicAdd(T.qsum + 2 * ch.x, s_q[0][threadIdx.x >> 5]);
    if (B.closed) atomicAdd(T.qsum + 2 * ch.x + 1, s_q[1][threadIdx.x >> 5]);
  }

  // ---- spreading: exact fixed point, one 32-bit word per staged node and
  // component; components 0 and 1 in one pass (buffers A and B), component 2
  // in a second (A), each pass flushed with float4 global atomics ----------
  if (SPREAD && !REC) {
    const float cl = area * sc.cl_scale;
    int* accA = reinterpret_cast<int*>(bufA);
    int* accB = reinterpret_cast<int*>(bufB);
    if (fit) {
      if (VEL) __syncthreads();   // the velocity phase is done with the buffers
      for (int q = threadIdx.x; q < ngroups; q += blockDim.x) {
        reinterpret_cast<int4*>(accA)[q] = make_int4(0, 0, 0, 0);
        reinterpret_cast<int4*>(accB)[q] = make_int4(0, 0, 0, 0);
      }
    }
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
      const int c0 = 2 * pass, nc = pass == 0 ? 2 : 1;   // components c0 .. c0 + nc - 1
      const float F0 = pass == 0 ? Fl[0] : Fl[2];
      const float F1 = Fl[1];
      if (fit) {
        // per component, the block's bound on |c_l phi F| from the bound on
        // |phi| (non-negative floats order as their bit patterns)
        float b0 = mine ? fabsf(cl * F0) * phi_bound_all : 0.f;
        float b1 = (mine && nc == 2) ? fabsf(cl * F1) * phi_bound_all : 0.f;
        if (!(b0 <= 3.0e38f)) b0 = __int_as_float(0x7f800000);
        if (!(b1 <= 3.0e38f)) b1 = __int_as_float(0x7f800000);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          b0 = fmaxf(b0, __shfl_xor_sync(0xffffffffu, b0, o));
          b1 = fmaxf(b1, __shfl_xor_sync(0xffffffffu, b1, o));
        }
        if ((threadIdx.x & 31) == 0) {
          atomicMax(&s_bmax[c0], __float_as_int(b0));
          if (nc == 2) atomicMax(&s_bmax[1], __float_as_int(b1));
        }
        __syncthreads();   // also: the buffers are zero
      }
      float inv[2] = {0.f, 0.f};
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        if (j >= nc) break;
        const int comp = j == 0 ? c0 : 1;
        const float coef = cl * (j == 0 ? F0 : F1);
        int cc[3];
        DirW X, Y, Z;
        if (mine) {
          float t3[3];
          locate(tc, comp, B.G, cc, t3);
          dir_weights(t3[0], sc.kappa, X);
          dir_weights(t3[1], sc.kappa, Y);
          dir_weights(t3[2], sc.kappa, Z);
        }
        if (fit) {
          const float bm = __int_as_float(s_bmax[comp]);
          if (!(bm <= 3.0e38f)) {
            if (threadIdx.x == 0) atomicOr(T.err, ERR_NONFINITE);
            continue;   // uniform over the block
          }
          if (bm == 0.f) continue;   // nothing to spread for this component
          // scale 2^k with every contribution below 2^22: a node takes at most
          // MT <= 256 of them, so the sum stays below 2^30
          const int k = min(22 - (ilogbf(bm) + 1), 120);
          inv[j] = pow2f(-max(k, -126));
          if (mine && coef != 0.f)
            mls_spread_fixed1(j == 0 ? accA : accB, SR.at(cc), X, Y, Z, coef * pow2f(max(k, -126)));
        } else if (mine) {
          spread_global(comp == 0 ? fx : (comp == 1 ? fy : fz), g, cc[0], cc[1], cc[2], X, Y, Z,
                        coef);
        }
      }
      if (fit) {
        __syncthreads();
        float* fa = c0 == 0 ? fx : fz;
        for (int q = threadIdx.x; q < ngroups; q += blockDim.x) {
          const int4 a = reinterpret_cast<const int4*>(accA)[q];
          const int4 b = nc == 2 ? reinterpret_cast<const int4*>(accB)[q] : make_int4(0, 0, 0, 0);
          const bool na = (a.x | a.y | a.z | a.w) != 0, nb = (b.x | b.y | b.z | b.w) != 0;
          if (!na && !nb) continue;
          if (na) reinterpret_cast<int4*>(accA)[q] = make_int4(0, 0, 0, 0);
          if (nb) reinterpret_cast<int4*>(accB)[q] = make_int4(0, 0, 0, 0);
          const float4 va = make_float4((float)a.x * inv[0], (float)a.y * inv[0], (float)a.z * inv[0],
                                        (float)a.w * inv[0]);
          const float4 vb = make_float4((float)b.x * inv[1], (float)b.y * inv[1], (float)b.z * inv[1],
                                        (float)b.w * inv[1]);
          if (vec4) {
            if (na) atomicAdd(reinterpret_cast<float4*>(fa + RT.node(q, 0)), va);
            if (nb) atomicAdd(reinterpret_cast<float4*>(fy + RT.node(q, 0)), vb);
          } else {
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
              const size_t o = RT.node(q, jj);
              const float xa = jj == 0 ? va.x : (jj == 1 ? va.y : (jj == 2 ? va.z : va.w));
              const float xb = jj == 0 ? vb.x : (jj == 1 ? vb.y : (jj == 2 ? vb.z : vb.w));
              if (xa != 0.f) atomicAdd(fa + o, xa);
              if (xb != 0.f) atomicAdd(fy + o, xb);
            }
          }
          const int r = s_grow[q];
          atomicMin(&s_nzlo[r], q);
          atomicMax(&s_nzhi[r], q);
        }
        __syncthreads();   // buffers zero again before the next pass
      }
    }
    if (record) {
      // footprint for the next step's clear: per row the x-range of the groups
      // that received a nonzero spread (staged), the bounding box (flag 1)
      // otherwise
      const int gc = B.chunk_off + ch.w;
      if (fit) {
        for (int r = threadIdx.x; r < sy * sz; r += blockDim.x) {
          int2 e = make_int2(0, 0);
          if (s_xmax[r] > 0 && s_nzlo[r] <= s_nzhi[r]) {
            const int L = min(4 * (s_nzhi[r] - s_nzlo[r] + 1), g.n[0]);
            const int go = s_gofs[s_nzlo[r]], x0 = go % g.n[0];
            e = make_int2(go - x0, x0 | (L << 16));
          }
          T.rowmap[(size_t)gc * kMaxRows + r] = e;
        }
      }
      if (threadIdx.x == 0) {
        T.boxes[2 * gc] = make_int4(xlo, ylo, zlo, fit ? (vec4 ? 2 : 0) : 1);
        T.boxes[2 * gc + 1] = make_int4(min(sx, g.n[0]), min(sy, g.n[1]), min(sz, g.n[2]),
                                        fit ? sy * sz : 0);
      }
    }
  }
}

// Zero the force fields on the footprint each marker block recorded in its
// last spread: its rows' nonzero x-ranges, or its bounding box when it took
// the global path.  Zeroing more than the footprint is harmless (everything
// nonzero belongs to some recorded footprint), so vector rows are widened to
// whole 32-byte sectors when nx allows, which avoids partial-sector writes
// (widening further to 64 bytes measured slower: more bytes written).
__global__ void __launch_bounds__(256) clear_kernel(DeviceTables T, Grid g, float* __restrict__ fx,
                                                    float* __restrict__ fy, float* __restrict__ fz,
                                                    int vec4, const int4* __restrict__ chunks,
                                                    int4* __restrict__ boxes,
                                                    const int2* __restrict__ rowmap, int max_rows) {
  // the marker kernel launched after this one may start at once: it waits
  // for this grid's completion before it touches what this grid writes
  asm volatile("griddepcontrol.launch_dependents;");
  // the first chunk of each body also zeroes the body's fixed-point sums
  if (threadIdx.x == 0) {
    const int4 ch = chunks[blockIdx.x];
    if (ch.w == 0) {
      T.qsum[2 * ch.x] = 0ull;
      T.qsum[2 * ch.x + 1] = 0ull;
    }
  }
  const int4 lo = boxes[2 * blockIdx.x];
  const int4 sz = boxes[2 * blockIdx.x + 1];
  if (sz.x <= 0 || sz.y <= 0 || sz.z <= 0) return;
  const int nx = g.n[0];
  // float4 stores only for rows recorded in whole float4 groups
  vec4 = vec4 && lo.w == 2;
  if (lo.w == 1) {
    const long long N = (long long)sz.x * sz.y * sz.z;
    const int sxy = sz.x * sz.y;
    for (long long idx = threadIdx.x; idx < N; idx += blockDim.x) {
      const int k = (int)(idx / sxy), rem = (int)(idx - (long long)k * sxy), j = rem / sz.x,
                i = rem - j * sz.x;
      const size_t o = ((size_t)wrap(lo.z + k, g.n[2]) * g.n[1] + wrap(lo.y + j, g.n[1])) * nx +
                       wrap(lo.x + i, nx);
      fx[o] = 0.f;
      fy[o] = 0.f;
      fz[o] = 0.f;
    }
  } else {
    const int nrows = sz.w;
    const int2* rm = rowmap + (size_t)blockIdx.x * max_rows;
    const int al = nx % 8 == 0 ? 8 : 4;   // widening, in floats
    // each warp takes 32 rows at a time: one coalesced load of their records,
    // then its four 8-lane groups clear 8 rows each, the records passed by
    // shuffles (eight lanes per row: each store instruction of a warp covers
    // four rows with one contiguous 128-byte span each)
    const int lane = threadIdx.x & 31, sub = lane & 7, grp = lane >> 3;
    for (int r0 = (threadIdx.x >> 5) * 32; r0 < nrows; r0 += blockDim.x) {
      const int2 mine = r0 + lane < nrows ? rm[r0 + lane] : make_int2(0, 0);
#pragma unroll 1
      for (int j = 0; j < 8; ++j) {
        const int src = 8 * grp + j;
        const int ex = __shfl_sync(0xffffffffu, mine.x, src);
        const int ey = __shfl_sync(0xffffffffu, mine.y, src);
        int L = ey >> 16, x0 = ey & 0xFFFF;  // (row base, first x wrapped | length << 16)
        if (L <= 0) continue;
        if (vec4) {
          L = min((L + (x0 & (al - 1)) + al - 1) & ~(al - 1), nx);
          x0 &= ~(al - 1);
          for (int q = 4 * sub; q < L; q += 32) {
            int xg = x0 + q;
            if (xg >= nx) xg -= nx;
            const size_t o = (size_t)ex + xg;
            const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
            *reinterpret_cast<float4*>(fx + o) = z4;
            *reinterpret_cast<float4*>(fy + o) = z4;
            *reinterpret_cast<float4*>(fz + o) = z4;
          }
        } else {
          for (int q = sub; q < L; q += 8) {
            int xg = x0 + q;
            if (xg >= nx) xg -= nx;
            const size_t o = (size_t)ex + xg;
            fx[o] = 0.f;
            fy[o] = 0.f;
            fz[o] = 0.f;
          }
        }
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) boxes[2 * blockIdx.x + 1] = make_int4(0, 0, 0, 0);
}

// (A, V) in float64 and the global-term coefficients from the fixed-point sums
__global__ void measure_finalize_kernel(DeviceTables T, int32_t nb) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const BodyDev B = T.body[b];
  const unsigned long long qa = T.qsum[2 * b], qv = T.qsum[2 * b + 1];
  T.meas[2 * b] = (double)(long long)qa / (double)B.sA;
  T.meas[2 * b + 1] = B.closed ? (double)(long long)qv / (double)B.sV : 0.0;
  T.coef[b] = body_coef(B, qa, qv);
}

// null (unused) pointers count as aligned
inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

template <int MT, bool M, bool I, bool P, bool S, bool R>
cudaError_t launch_mt(ibm_ctx* c, const float* x, const float* v, const float* u, const float* vv,
                      const float* w, const float* pr, const float* accel, float* U, float* Fm,
                      const float* Fm_in, float* Fext, float* fx, float* fy, float* fz,
                      int record, int tmode, const DeviceTables* tab, int cache, bool pdl) {
  const size_t smem = (I || P || (S && !R)) ? marker_smem_bytes(MT) : 0;
  const int vec4 = c->vec4 && aligned16(u) && aligned16(vv) && aligned16(w) && aligned16(pr) &&
                   aligned16(fx) && aligned16(fy) && aligned16(fz);
  // pdl: launched as the programmatic dependent of the footprint clear just
  // before it on the stream (it may start once every clear block runs)
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)c->n_chunks);
  cfg.blockDim = dim3(MT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = c->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, marker_kernel<MT, M, I, P, S, R>, tab ? *tab : c->d, c->grid,
                            c->sc, (int32_t)c->V, (int32_t)c->F, x, v, u, vv, w, pr, accel, U,
                            Fm, Fm_in, Fext, fx, fy, fz, record, vec4, c->td, tmode,
                            c->phi_bound, cache, c->fc_tab, c->fc_face);
}

// the marker kernel for the context's patch size (128 or 256 faces per block)
template <bool M, bool I, bool P, bool S, bool R = false>
cudaError_t launch_t(ibm_ctx* c, const float* x, const float* v, const float* u, const float* vv,
                     const float* w, const float* pr, const float* accel, float* U, float* Fm,
                     const float* Fm_in, float* Fext, float* fx, float* fy, float* fz,
                     int record, int tmode = 0, const DeviceTables* tab = nullptr, int cache = 0,
                     bool pdl = false) {
  if (c->n_chunks == 0) return cudaSuccess;
  if (c->marker_patch == 128)
    return launch_mt<128, M, I, P, S, R>(c, x, v, u, vv, w, pr, accel, U, Fm, Fm_in, Fext, fx, fy,
                                         fz, record, tmode, tab, cache, pdl);
  return launch_mt<kMT, M, I, P, S, R>(c, x, v, u, vv, w, pr, accel, U, Fm, Fm_in, Fext, fx, fy,
                                       fz, record, tmode, tab, cache, pdl);
}

}  // namespace

cudaError_t set_marker_smem_limit() {
  cudaError_t e = cudaSuccess;
#define SET(M, I, P, S, R)                                                                   \
  if (e == cudaSuccess)                                                                      \
    e = cudaFuncSetAttribute(marker_kernel<kMT, M, I, P, S, R>,                              \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, kMarkerSmemBytes);  \
  if (e == cudaSuccess)                                                                      \
    e = cudaFuncSetAttribute(marker_kernel<128, M, I, P, S, R>,                              \
                             cudaFuncAttributeMaxDynamicSharedMemorySize,                    \
                             marker_smem_bytes(128));
  SET(true, true, true, true, false)
  SET(true, false, true, false, false)
  SET(false, true, true, false, false)
  SET(false, true, false, false, false)
  SET(false, false, true, false, false)
  SET(false, false, false, true, false)
  SET(false, true, false, true, false)
  SET(true, true, true, true, true)
  SET(false, true, false, true, true)
#undef SET
  return e;
}

cudaError_t launch_mls(ibm_ctx* c, const float* x, const float* v, const float* u,
                       const float* vv, const float* w, const float* pr, const float* accel,
                       float* U, float* Fm, const float* Fm_in, float* Fext, float* fx, float* fy,
                       float* fz, bool measure, bool interp, bool probe, bool spread,
                       bool record_box, bool after_clear) {
  const int rb = record_box ? 1 : 0;
#define L(M, I, P, S) \
  launch_t<M, I, P, S>(c, x, v, u, vv, w, pr, accel, U, Fm, Fm_in, Fext, fx, fy, fz, rb)
  if (measure && interp && probe && spread)
    return launch_t<true, true, true, true>(c, x, v, u, vv, w, pr, accel, U, Fm, Fm_in, Fext, fx,
                                            fy, fz, rb, 0, nullptr, 0, after_clear);
  if (measure && !interp && !probe && !spread) return L(true, false, false, false);
  if (measure && !interp && probe && !spread) return L(true, false, true, false);
  if (!measure && interp && probe && !spread) return L(false, true, true, false);
  if (!measure && interp && !probe && !spread) return L(false, true, false, false);
  if (!measure && !interp && probe && !spread) return L(false, false, true, false);
  if (!measure && !interp && !probe && spread) return L(false, false, false, true);
  if (!measure && interp && !probe && spread) return L(false, true, false, true);
#undef L
  return cudaErrorInvalidValue;
}

cudaError_t launch_mls_records(ibm_ctx* c, const float* x, const float* v, const float* u,
                               const float* vv, const float* w, const float* p,
                               const float* accel, const float* Fm_in, float* Fext, bool measure,
                               bool probe, bool accumulate) {
  const int tm = accumulate ? 2 : 1;
  if (measure && probe)   // the step: body sums, interpolation, traction, records
    return launch_t<true, true, true, true, true>(c, x, v, u, vv, w, p, accel, nullptr, nullptr,
                                                  nullptr, Fext, nullptr, nullptr, nullptr, 0, tm);
  if (!measure && !probe && u)   // the coupled forcing: interpolation and records
    return launch_t<false, true, false, true, true>(c, x, v, u, vv, w, nullptr, nullptr, nullptr,
                                                    nullptr, nullptr, nullptr, nullptr, nullptr,
                                                    nullptr, 0, tm);
  if (!measure && !probe && Fm_in)   // given marker forces
    return launch_t<false, false, false, true, true>(c, x, nullptr, nullptr, nullptr, nullptr,
                                                     nullptr, nullptr, nullptr, nullptr, Fm_in,
                                                     nullptr, nullptr, nullptr, nullptr, 0, tm);
  return cudaErrorInvalidValue;
}

cudaError_t zero_body_sums(ibm_ctx* c) {
  if (c->B == 0) return cudaSuccess;
  return cudaMemsetAsync(c->d.qsum, 0, sizeof(unsigned long long) * 2 * c->B, c->stream);
}

cudaError_t launch_measure_finalize(ibm_ctx* c) {
  if (c->B == 0) return cudaSuccess;
  measure_finalize_kernel<<<(unsigned)((c->B + 127) / 128), 128, 0, c->stream>>>(c->d,
                                                                               (int32_t)c->B);
  return cudaGetLastError();
}

cudaError_t launch_clear(ibm_ctx* c, float* fx, float* fy, float* fz) {
  if (c->n_chunks == 0) return cudaSuccess;
  const int vec4 = c->vec4 && aligned16(fx) && aligned16(fy) && aligned16(fz);
  clear_kernel<<<c->n_chunks, 256, 0, c->stream>>>(c->d, c->grid, fx, fy, fz, vec4, c->d.chunks,
                                                  c->d.boxes, c->d.rowmap, kMaxRows);
  return cudaGetLastError();
}

// The coupled forcing of substep `substep` (interpolation of u* and spread
// at the centroids of x): footprints recorded in the flow's own record (the
// step's record is left alone), the previous substep's footprint cleared
// first (substep 0: the caller zeroes the fields), and the face geometry and
// row tables saved in substep 0 and loaded in substeps 1 and 2.
cudaError_t launch_forcing(ibm_ctx* c, int substep, const float* x, const float* xv,
                           const float* u, const float* vv, const float* w, float* fx, float* fy,
                           float* fz) {
  if (c->n_chunks == 0) return cudaSuccess;
  DeviceTables t = c->d;
  t.boxes = c->fc_boxes;
  t.rowmap = c->fc_rowmap;
  if (substep > 0) {
    const int vec4 = c->vec4 && aligned16(fx) && aligned16(fy) && aligned16(fz);
    clear_kernel<<<c->n_chunks, 256, 0, c->stream>>>(t, c->grid, fx, fy, fz, vec4, c->d.chunks,
                                                    t.boxes, t.rowmap, kMaxRows);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return launch_t<false, true, false, true>(c, x, xv, u, vv, w, nullptr, nullptr, nullptr, nullptr,
                                            nullptr, nullptr, fx, fy, fz, 1, 0, &t,
                                            substep == 0 ? 1 : 2);
}

}  // namespace ibm
