// Tile-owned spreading of the marker forces onto the staggered grid (Sec. 2.2,
// Eq. mls_cl: f_i^k = sum over the markers l whose support holds node k of
// c_l phi_k^l F_i^l), deterministic and without global atomics on the fields.
//
// The marker kernel (record mode) writes one record per marker (centroid in
// cells, c_l F) and counts, per tile of kTX x kTY x kTZ grid nodes, the markers
// whose centroid supports reach it (the union over the three components of the
// 3x3x3 nearest-node supports: nodes f-1 .. f+2 per direction), with the
// largest |c_l F| per component.  Then:
//   tile_scan_kernel    every tile once: reached tiles get a range in the
//                       marker list and are listed, with the tiles the previous
//                       clear-mode call reached and this one does not,
//   tile_fill_kernel    each marker writes its id into the ranges of its tiles,
//   tile_spread_kernel  one block per listed tile: every listed marker adds
//                       c_l phi F to the tile's nodes it supports, in exact
//                       fixed point in shared memory (a power-of-two scale per
//                       tile and component, so the sum does not depend on the
//                       order); the tile then stores every 8-node x-segment that
//                       received contributions or that the previous clear-mode
//                       call left nonzero (a bit mask per tile), with plain
//                       stores: each node is written by exactly one block, once.
// A clear-mode call thereby leaves exactly this call's forces in the fields
// (no separate clear, no read of the fields); accumulate mode adds the tile's
// nonzero nodes to the fields' values (read, add, store: still one owner per
// node).  The epoch of clear-mode calls is kept on the device, so a captured
// sequence of steps needs no host state.
#include <cuda_runtime.h>
#include <limits.h>
#include <math.h>

#include <algorithm>

#include "ibm_internal.cuh"

namespace ibm {
namespace {

// closed-form MLS factors of one direction (the same as the marker kernel's:
// normalised weights a_s and b_s = a_s beta_s of the three nodes at offsets
// -1, 0, +1 from the nearest node, for the fractional offset tp in [-1/2, 1/2))
__device__ __forceinline__ void dir_factors(float tp, float kappa, float (&a)[3], float (&b)[3]) {
  const float rm = __expf(-kappa * fmaf(2.f, tp, 1.f)), rp = __expf(-kappa * fmaf(-2.f, tp, 1.f));
  const float invS = __fdividef(1.f, 1.f + rm + rp);
  const float a0 = rm * invS, a1 = invS, a2 = rp * invS;
  const float d0 = -1.f - tp, d1 = -tp, d2 = 1.f - tp;
  const float mu = a0 * d0 + a1 * d1 + a2 * d2;
  const float e0 = d0 - mu, e1 = d1 - mu, e2 = d2 - mu;
  const float s2 = a0 * e0 * e0 + a1 * e1 * e1 + a2 * e2 * e2;
  const float r = __fdividef(mu, s2);
  a[0] = a0; a[1] = a1; a[2] = a2;
  b[0] = a0 * r * e0; b[1] = a1 * r * e1; b[2] = a2 * r * e2;
}

// begin a call: the epoch (clear mode), the list length, the pair total, and
// the fixed-point body sums of the marker kernel
__global__ void tile_begin_kernel(TileDev td, unsigned long long* qsum, int nq, int accumulate) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    if (!accumulate) td.state[TS_EPOCH] += 1;
    td.state[TS_LEN] = 0;
    td.state[TS_PAIRS] = 0;
  }
  if (qsum && i < nq) qsum[i] = 0ull;
}

// block-wide exclusive scan of v (blockDim.x multiple of 32, <= 1024); returns
// the exclusive prefix, *total the block's sum (s_warp: 32 ints of scratch)
__device__ __forceinline__ int block_scan(int v, int* s_warp, int* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_warp[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int w = lane < nw ? s_warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < nw) s_warp[lane] = w;
  }
  __syncthreads();
  const int ex = (wid ? s_warp[wid - 1] : 0) + incl - v;
  *total = s_warp[nw - 1];
  __syncthreads();
  return ex;
}

// every tile once: the tiles that markers reach in this call get a range in
// the marker list and are listed; in clear mode so are the tiles that the
// previous clear-mode call listed and this one does not (their segments are
// zeroed), and the reached tiles take this call's epoch
template <bool CLEAR>
__global__ void __launch_bounds__(1024) tile_scan_kernel(TileDev td) {
  __shared__ int s_warp[32];
  __shared__ int s_pbase, s_lbase;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = t < td.n_tiles;
  const int cnt = valid ? td.count[t] : 0;
  bool listed = cnt > 0;
  if (CLEAR && valid) {
    const int e = td.state[TS_EPOCH];
    const int last = td.epoch[t];
    listed = listed || last == e - 1;
    if (cnt > 0) td.epoch[t] = e;
  }
  int ptot, ltot;
  const int pex = block_scan(cnt, s_warp, &ptot);
  const int lex = block_scan(listed ? 1 : 0, s_warp, &ltot);
  if (threadIdx.x == 0) {
    s_pbase = ptot ? atomicAdd(td.state + TS_PAIRS, ptot) : 0;
    s_lbase = ltot ? atomicAdd(td.state + TS_LEN, ltot) : 0;
  }
  __syncthreads();
  if (listed) {
    td.active[0][s_lbase + lex] = t;
    td.off[t] = s_pbase + pex;
    td.cur[t] = s_pbase + pex;
  }
}

// every marker with a record writes its id into the lists of its tiles (the
// same tiles, from the same record, as the marker kernel counted)
__global__ void __launch_bounds__(256) tile_fill_kernel(DeviceTables T, TileDev td, Grid g,
                                                        int32_t F) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  const float4 r0 = td.rec[2 * (size_t)f];
  const int b = __float_as_int(r0.w);
  if (b < 0) return;
  const int G0 = __ldg(&T.body[b].G[0]), G1 = __ldg(&T.body[b].G[1]), G2 = __ldg(&T.body[b].G[2]);
  int tx[3], ty[3], tz[3];
  const int nx_ = tiles_along(G0 + (int)floorf(r0.x), g.n[0], kTX, tx);
  const int ny_ = tiles_along(G1 + (int)floorf(r0.y), g.n[1], kTY, ty);
  const int nz_ = tiles_along(G2 + (int)floorf(r0.z), g.n[2], kTZ, tz);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int d = 0; d < 3; ++d)
        if (a < nz_ && c < ny_ && d < nx_) {
          const int t = (tz[a] * td.nt[1] + ty[c]) * td.nt[0] + tx[d];
          td.mlist[atomicAdd(td.cur + t, 1)] = f;
        }
}

// One block per listed tile (a persistent grid walks the list).  A thread per
// (listed marker, component) adds c_l phi F to the tile's nodes in exact fixed
// point: q = c_l phi F 2^k, its float value rounded to an integer, split into
// hi = floor(q / 2^16) and lo = q - 2^16 hi in [0, 2^16], each summed with a
// 32-bit shared atomic (lo as unsigned).  With n markers listed and
// |q| <= min(2^38, 2^45 / n_pow2) the hi sums stay below 2^30 and the lo sums
// below 2^32 for n < 2^16; the node's value 2^16 sum(hi) + sum(lo) is exact
// and does not depend on the order.  2^k comes from the tile's largest |c_l F|
// (recorded by the marker kernel) and the bound on |phi|.  The x-segments of 8
// nodes that receive contributions, and in clear mode those the previous call
// left nonzero, are then stored (8 threads per segment) and their
// accumulators zeroed again for the block's next tile.
template <bool CLEAR>
__global__ void __launch_bounds__(kTileThreads) tile_spread_kernel(
    DeviceTables T, TileDev td, Grid g, float kappa, float phi_bound, float* __restrict__ fx,
    float* __restrict__ fy, float* __restrict__ fz) {
  __shared__ int s_hi[3][kTileNodes];
  __shared__ unsigned s_lo[3][kTileNodes];
  __shared__ uint32_t s_prev[12], s_new[12];
  __shared__ unsigned char s_touch[3 * kTileNodes / 8];   // segment received a contribution
  __shared__ unsigned short s_seg[3 * kTileNodes / 8];
  __shared__ unsigned s_tmax[3];
  __shared__ int s_m0, s_m1, s_nseg;
  const int lane = threadIdx.x & 31;
  for (int q = threadIdx.x; q < 3 * kTileNodes / 4; q += blockDim.x) {
    reinterpret_cast<int4*>(&s_hi[0][0])[q] = make_int4(0, 0, 0, 0);
    reinterpret_cast<int4*>(&s_lo[0][0])[q] = make_int4(0, 0, 0, 0);
  }
  for (int q = threadIdx.x; q < 3 * kTileNodes / 8; q += blockDim.x) s_touch[q] = 0;
  if (threadIdx.x == 0) s_nseg = 0;
  const int L = td.state[TS_LEN];
  for (int item = blockIdx.x; item < L; item += gridDim.x) {
    const int t = td.active[0][item];
    const int tx = t % td.nt[0], ty = (t / td.nt[0]) % td.nt[1], tz = t / (td.nt[0] * td.nt[1]);
    const int X0 = tx * kTX, Y0 = ty * kTY, Z0 = tz * kTZ;
    const int ex = min(kTX, g.n[0] - X0), ey = min(kTY, g.n[1] - Y0), ez = min(kTZ, g.n[2] - Z0);
    if (threadIdx.x < 12) {
      s_prev[threadIdx.x] = CLEAR ? td.mask[12 * (size_t)t + threadIdx.x] : 0u;
      s_new[threadIdx.x] = 0u;
    }
    if (threadIdx.x == 0) {
      s_m0 = td.off[t];
      s_m1 = td.cur[t];
      td.count[t] = 0;   // ready for the next call
    }
    if (threadIdx.x < 3) {
      s_tmax[threadIdx.x] = td.tmax[4 * (size_t)t + threadIdx.x];
      td.tmax[4 * (size_t)t + threadIdx.x] = 0u;
    }
    __syncthreads();
    const int m0 = s_m0, n = s_m1 - s_m0;
    // scale 2^k per component with phi_bound * max|c_l F| * 2^k <= qcap
    int np2 = 1;
    while (np2 < n && np2 < (1 << 20)) np2 <<= 1;
    const float qcap = fminf(0x1p38f, __int_as_float((127 + 45) << 23) / (float)np2);
    float scale[3], inv_scale[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const float bm = __uint_as_float(s_tmax[i]) * phi_bound;
      scale[i] = 0.f;
      inv_scale[i] = 0.f;
      if (bm > 0.f && bm <= 3.0e38f) {
        const int k = max(min(ilogbf(qcap) - (ilogbf(bm) + 1), 120), -120);
        scale[i] = __int_as_float((k + 127) << 23);
        inv_scale[i] = __int_as_float((127 - k) << 23);
      }
    }
    if (threadIdx.x == 0 && n >= 65536) atomicOr(T.err, ERR_TILE_DENSE);
    // contributions: thread q -> marker q / 3, component q % 3
    for (int q = threadIdx.x; q < 3 * n; q += blockDim.x) {
      const int jm = q / 3, i = q - 3 * jm;
      const int m = td.mlist[m0 + jm];
      const float4 r0 = td.rec[2 * (size_t)m];
      const float* r1 = reinterpret_cast<const float*>(td.rec + 2 * (size_t)m + 1);
      const float sc = i == 0 ? scale[0] : (i == 1 ? scale[1] : scale[2]);
      const float coef = __ldg(r1 + i) * sc;
      if (coef == 0.f) continue;
      const int b = __float_as_int(r0.w);
      const int G[3] = {__ldg(&T.body[b].G[0]), __ldg(&T.body[b].G[1]), __ldg(&T.body[b].G[2])};
      const float tc[3] = {r0.x, r0.y, r0.z};
      const int T0[3] = {X0, Y0, Z0}, EX[3] = {ex, ey, ez};
      float a[3][3], bb[3][3], uf[3];
      int loc[3][3];
      bool reach = true;   // this component's support meets the tile
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const float uu = tc[d] - (d == i ? 0.f : 0.5f);
        const float cc = floorf(uu + 0.5f);
        uf[d] = uu - cc;
        const int c0 = G[d] + (int)cc - 1;
        bool any = false;
#pragma unroll
        for (int s2 = 0; s2 < 3; ++s2) {
          const int l = wrap_any(c0 + s2, g.n[d]) - T0[d];
          loc[d][s2] = (l >= 0 && l < EX[d]) ? l : -1;
          any = any || loc[d][s2] >= 0;
        }
        reach = reach && any;
      }
      if (!reach) continue;
#pragma unroll
      for (int d = 0; d < 3; ++d) dir_factors(uf[d], kappa, a[d], bb[d]);
      int* hi = i == 0 ? s_hi[0] : (i == 1 ? s_hi[1] : s_hi[2]);
      unsigned* lo = i == 0 ? s_lo[0] : (i == 1 ? s_lo[1] : s_lo[2]);
      // the x-segments (0, 1) of a row that this marker touches
      bool seg0 = false, seg1 = false;
#pragma unroll
      for (int sx = 0; sx < 3; ++sx) {
        seg0 = seg0 || (loc[0][sx] >= 0 && loc[0][sx] < 8);
        seg1 = seg1 || loc[0][sx] >= 8;
      }
#pragma unroll
      for (int sz = 0; sz < 3; ++sz) {
        if (loc[2][sz] < 0) continue;
#pragma unroll
        for (int sy = 0; sy < 3; ++sy) {
          if (loc[1][sy] < 0) continue;
          const float ay = a[1][sy], by = bb[1][sy], az = a[2][sz], bz = bb[2][sz];
          const float t0 = ay * az * coef, t1 = (by * az + ay * bz) * coef;
          const int rowi = loc[2][sz] * kTY + loc[1][sy];
          const int row = rowi * kTX;
#pragma unroll
          for (int sx = 0; sx < 3; ++sx) {
            if (loc[0][sx] < 0) continue;
            const float val = rintf((a[0][sx] - bb[0][sx]) * t0 - a[0][sx] * t1);
            const float hf = floorf(val * (1.f / 65536.f));
            atomicAdd(hi + row + loc[0][sx], (int)hf);
            atomicAdd(lo + row + loc[0][sx], (unsigned)fmaf(-hf, 65536.f, val));
          }
          // flags set with plain stores (every writer stores 1)
          if (seg0) s_touch[128 * i + 2 * rowi] = 1;
          if (seg1) s_touch[128 * i + 2 * rowi + 1] = 1;
        }
      }
    }
    __syncthreads();
    // segments to store: touched now, or (clear mode) nonzero after the last call
    for (int sg = threadIdx.x; sg < 3 * kTileNodes / 8; sg += blockDim.x) {
      const uint32_t bit = 1u << (sg & 31);
      if (s_touch[sg] || (s_prev[sg >> 5] & bit)) {
        s_seg[atomicAdd(&s_nseg, 1)] = (unsigned short)sg;
        s_touch[sg] = 0;
      }
    }
    __syncthreads();
    const int nseg = s_nseg;
    // 8 threads per segment; each warp handles 4 segments per pass, all
    // lanes take part in the ballot
    for (int base = (threadIdx.x >> 5) * 32; base < 8 * nseg; base += blockDim.x) {
      const int k = base + lane;
      const bool act = k < 8 * nseg;
      float val = 0.f;
      int i = 0, nid = 0;
      if (act) {
        const int sg = s_seg[k >> 3];
        i = sg >> 7;
        nid = ((sg & 127) << 3) + (k & 7);
        const long long S = (long long)s_hi[i][nid] * 65536ll + (long long)s_lo[i][nid];
        s_hi[i][nid] = 0;
        s_lo[i][nid] = 0u;
        const float inv = i == 0 ? inv_scale[0] : (i == 1 ? inv_scale[1] : inv_scale[2]);
        val = fmaf((float)(int)(S >> 32), 4294967296.f, (float)(unsigned)(S & 0xffffffffll)) * inv;
      }
      const unsigned bal = __ballot_sync(0xffffffffu, val != 0.f);
      if (act) {
        const int x = nid % kTX, y = (nid / kTX) % kTY, z = nid / (kTX * kTY);
        const bool inside = x < ex && y < ey && z < ez;
        float* fc = i == 0 ? fx : (i == 1 ? fy : fz);
        const size_t idx = ((size_t)(Z0 + z) * g.n[1] + (Y0 + y)) * g.n[0] + (X0 + x);
        if (CLEAR) {
          if (inside) fc[idx] = val;
          const bool seg_nz = ((bal >> (lane & ~7)) & 0xffu) != 0u;
          if (seg_nz && (lane & 7) == 0) {
            const int gs = 128 * i + (nid >> 3);
            atomicOr(&s_new[gs >> 5], 1u << (gs & 31));
          }
        } else if (inside && val != 0.f) {
          fc[idx] += val;
        }
      }
    }
    __syncthreads();
    if (CLEAR && threadIdx.x < 12) td.mask[12 * (size_t)t + threadIdx.x] = s_new[threadIdx.x];
    if (threadIdx.x == 0) s_nseg = 0;
    __syncthreads();
  }
}

}  // namespace

cudaError_t tile_spread_occupancy(int* blocks_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, tile_spread_kernel<true>,
                                                       kTileThreads, 0);
}

cudaError_t launch_tile_begin(ibm_ctx* c, bool accumulate, bool zero_sums) {
  const int nq = zero_sums ? 2 * (int)c->B : 0;
  const int blocks = (nq + 255) / 256 > 0 ? (nq + 255) / 256 : 1;
  tile_begin_kernel<<<blocks, 256, 0, c->stream>>>(c->td, zero_sums ? c->d.qsum : nullptr, nq,
                                                   accumulate ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_tile_spread(ibm_ctx* c, float* fx, float* fy, float* fz, bool accumulate) {
  if (c->F == 0) return cudaSuccess;
  const unsigned nb = (unsigned)((c->td.n_tiles + 1023) / 1024);
  if (accumulate)
    tile_scan_kernel<false><<<nb, 1024, 0, c->stream>>>(c->td);
  else
    tile_scan_kernel<true><<<nb, 1024, 0, c->stream>>>(c->td);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  tile_fill_kernel<<<(unsigned)((c->F + 255) / 256), 256, 0, c->stream>>>(c->d, c->td, c->grid,
                                                                         (int32_t)c->F);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (accumulate)
    tile_spread_kernel<false><<<c->tile_grid, kTileThreads, 0, c->stream>>>(
        c->d, c->td, c->grid, c->sc.kappa, c->phi_bound, fx, fy, fz);
  else
    tile_spread_kernel<true><<<c->tile_grid, kTileThreads, 0, c->stream>>>(
        c->d, c->td, c->grid, c->sc.kappa, c->phi_bound, fx, fy, fz);
  return cudaGetLastError();
}

}  // namespace ibm
