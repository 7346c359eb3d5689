// Allocation-free per-body surface area and enclosed volume.
//
// Each face's float32 area and signed tetrahedron volume are summed in
// float64 in a fixed order (per block, then per body in chunk order), so the
// result is deterministic; it agrees with the context's body measures (which
// quantise each face to 2^-39 of the body's rest value and sum integers) to
// about that resolution.  It needs no context and allocates nothing: its
// scratch (per-chunk partial sums and per-body arrival counters) lives in one
// file-scope device array of fixed size that every GPU loading the library
// holds until the process exits.
//
// Caller data is checked on the device before it is used for addressing: a
// body whose face range is reversed or negative, whose faces need more chunks
// than max_faces_per_body allows, or that holds a vertex id outside [0, V)
// gets (NaN, NaN); a body with no faces gets (0, 0).
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "ibm_internal.cuh"

namespace {

constexpr int kNaThreads = 256;                       // faces per block (chunk)
constexpr long long kNaMaxChunks = 65536;             // bodies x chunks per body
constexpr long long kNaMaxBodies = 65535;            // grid y limit
constexpr size_t kNaPartialBytes = 2 * sizeof(double) * kNaMaxChunks;
constexpr size_t kNaScratchBytes = kNaPartialBytes + sizeof(int) * kNaMaxBodies;  // 1.25 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaScratchBytes];

std::mutex g_na_mu;
void* g_na_ptr[64] = {nullptr};                      // device address of the scratch, per device

// Block (c, b) sums faces [face_off[b] + 256 c, ...) of body b; the last of
// the body's chunks to arrive adds the chunk partials in chunk order.
__global__ void __launch_bounds__(kNaThreads) measures_noalloc_kernel(
    const float* __restrict__ x, int32_t V, const int32_t* __restrict__ tri,
    const int32_t* __restrict__ face_off, const uint8_t* __restrict__ closed, int32_t max_chunks,
    double* __restrict__ out, unsigned char* scratch) {
  double* partial = reinterpret_cast<double*>(scratch);
  int* counter = reinterpret_cast<int*>(scratch + kNaPartialBytes);
  __shared__ double s_red[2][kNaThreads / 32];
  __shared__ int s_last;
  const int b = blockIdx.y, c = blockIdx.x;
  const int f0 = face_off[b], f1 = face_off[b + 1];
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  // whole-body outcomes decided by chunk 0 alone (uniform across the block)
  if (f0 < 0 || f1 < f0 || (long long)(f1 - f0) > (long long)max_chunks * kNaThreads) {
    if (c == 0 && threadIdx.x == 0) {
      out[2 * b] = nan;
      out[2 * b + 1] = nan;
    }
    return;
  }
  if (f1 == f0) {
    if (c == 0 && threadIdx.x == 0) {
      out[2 * b] = 0.0;
      out[2 * b + 1] = 0.0;
    }
    return;
  }
  const int n_chunk = (f1 - f0 + kNaThreads - 1) / kNaThreads;
  if (c >= n_chunk) return;                           // uniform across the block
  const bool is_closed = closed ? closed[b] != 0 : true;
  const int f = f0 + c * kNaThreads + threadIdx.x;
  double a = 0.0, vol = 0.0;
  if (f < f1) {
    const int ia = tri[3 * f], ib = tri[3 * f + 1], ic = tri[3 * f + 2];
    // an out-of-range vertex id is never dereferenced: the face contributes
    // NaN, which the sums carry to the body's output
    const bool bad = ia < 0 || ia >= V || ib < 0 || ib >= V || ic < 0 || ic >= V;
    float xa[3] = {0.f, 0.f, 0.f}, xb[3] = {0.f, 0.f, 0.f}, xc[3] = {0.f, 0.f, 0.f};
    if (!bad) {
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        xa[d] = x[d * V + ia];
        xb[d] = x[d * V + ib];
        xc[d] = x[d * V + ic];
      }
    }
    const float e1[3] = {xb[0] - xa[0], xb[1] - xa[1], xb[2] - xa[2]};
    const float e2[3] = {xc[0] - xa[0], xc[1] - xa[1], xc[2] - xa[2]};
    const float N[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                        e1[0] * e2[1] - e1[1] * e2[0]};
    a = (double)(0.5f * sqrtf(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]));
    if (is_closed)
      vol = (double)((xa[0] * (xb[1] * xc[2] - xb[2] * xc[1]) + xa[1] * (xb[2] * xc[0] - xb[0] * xc[2]) +
                      xa[2] * (xb[0] * xc[1] - xb[1] * xc[0])) * (1.f / 6.f));
    if (bad) {
      a = nan;
      vol = nan;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    vol += __shfl_down_sync(0xffffffffu, vol, o);
  }
  if ((threadIdx.x & 31) == 0) {
    s_red[0][threadIdx.x >> 5] = a;
    s_red[1][threadIdx.x >> 5] = vol;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0.0, sv = 0.0;
    for (int k = 0; k < kNaThreads / 32; ++k) {
      sa += s_red[0][k];
      sv += s_red[1][k];
    }
    const size_t slot = (size_t)b * max_chunks + c;
    partial[2 * slot] = sa;
    partial[2 * slot + 1] = sv;
    __threadfence();
    s_last = (atomicAdd(counter + b, 1) == n_chunk - 1);
  }
  __syncthreads();
  if (s_last && threadIdx.x == 0) {
    __threadfence();
    const volatile double* P = partial;
    double ta = 0.0, tv = 0.0;
    for (int k = 0; k < n_chunk; ++k) {
      ta += P[2 * ((size_t)b * max_chunks + k)];
      tv += P[2 * ((size_t)b * max_chunks + k) + 1];
    }
    out[2 * b] = ta;
    out[2 * b + 1] = is_closed ? tv : (ta == ta ? 0.0 : nan);
    counter[b] = 0;
  }
}

ibm_status na_fail(ibm_status s, const std::string& m) {
  ibm::set_global_error(m);   // reported by ibm_last_error(NULL)
  return s;
}

}  // namespace

extern "C" ibm_status ibm_body_measures_noalloc(const float* x, int64_t n_vert, const int32_t* tri,
                                                const int32_t* face_off, int32_t n_bodies,
                                                int32_t max_faces_per_body, const uint8_t* closed,
                                                double* out, void* stream) {
  if (!x || !tri || !face_off || !out || n_vert <= 0 || n_bodies <= 0 || max_faces_per_body <= 0)
    return na_fail(IBM_ERR_INVALID_ARG, "ibm_body_measures_noalloc: null pointer or non-positive size");
  if (n_vert >= (1ll << 31) / 3)
    return na_fail(IBM_ERR_UNSUPPORTED, "ibm_body_measures_noalloc: too many vertices");
  const long long max_chunks = (max_faces_per_body + kNaThreads - 1) / kNaThreads;
  if (n_bodies > kNaMaxBodies || (long long)n_bodies * max_chunks > kNaMaxChunks)
    return na_fail(IBM_ERR_UNSUPPORTED,
                   "ibm_body_measures_noalloc: bodies x ceil(max_faces_per_body / 256) exceeds the "
                   "static scratch (65536 chunks, 65535 bodies)");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64)
    return na_fail(IBM_ERR_CUDA, std::string("ibm_body_measures_noalloc: cudaGetDevice: ") +
                                     cudaGetErrorString(e));
  void* scratch = nullptr;
  {
    // set-up, once per device, with that device current: the host-side name
    // of the array is not a device address, so ask the runtime for it
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
      e = cudaGetSymbolAddress(&g_na_ptr[dev], g_noalloc_scratch);
      if (e != cudaSuccess) {
        g_na_ptr[dev] = nullptr;
        ibm::set_global_error(std::string("ibm_body_measures_noalloc: cudaGetSymbolAddress: ") +
                              cudaGetErrorString(e));
        return IBM_ERR_CUDA;
      }
    }
    scratch = g_na_ptr[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the arrival counters must start at zero
  e = cudaMemsetAsync(static_cast<unsigned char*>(scratch) + kNaPartialBytes, 0,
                      sizeof(int) * (size_t)n_bodies, s);
  if (e == cudaSuccess) {
    measures_noalloc_kernel<<<dim3((unsigned)max_chunks, (unsigned)n_bodies), kNaThreads, 0, s>>>(
        x, (int32_t)n_vert, tri, face_off, closed, (int32_t)max_chunks, out,
        static_cast<unsigned char*>(scratch));
    e = cudaGetLastError();
  }
  if (e != cudaSuccess)
    return na_fail(IBM_ERR_CUDA, std::string("ibm_body_measures_noalloc: ") + cudaGetErrorString(e));
  return IBM_OK;
}
