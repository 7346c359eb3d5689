// Internal device-side layout shared by the host builder and the kernels of
// the GB300 IP + MLS-IBM library.  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ibm.h"

namespace ibm {

// ---------------------------------------------------------------------------
// per-body record (one per body, read by every kernel through the work lists)
// ---------------------------------------------------------------------------
struct BodyDev {
  int32_t v_off, f_off, e_off, topo;   // global offsets, topology id
  int32_t nv, nf, ne, closed;
  int32_t G[3];                        // floor(origin_d / h_d)
  int32_t chunk_off;                   // first marker chunk of this body
  float frac[3];                       // origin_d / h_d - G_d, in [0, 1)
  int32_t n_chunk;
  float ks, kb, ka, kA, kv, inv_mass;  // elastic constants, 1/m
  int32_t work_off;                    // first force-kernel work item (patch) of this body
  int32_t pad1;
  double A0, V0;                       // rest area and volume (float64)
  double fracd[3];                     // frac in float64 (the float64 interpolation option)
  // Exact fixed-point body sums: a face's area (volume) contributes
  // q = rint(value * sA) (sV), a power of two chosen from A0 (V0), and the
  // q are summed with 64-bit integer atomics, independent of order.
  int64_t qA0, qV0;                    // rest area and volume in fixed point
  float sA, sV;                        // 2^eA, 2^eV
  float cA_unit, cV_unit;              // k_A / (sA A0), k_v / (sV V0)
  float qlim;                          // per-face bound on |q|: 2^62 / n_faces
  int32_t varied;                      // 1: per-element multipliers kse, kbe, kaf apply
};

// per distinct mesh topology (shared by every body with the same faces)
struct TopoDev {
  int32_t nv, nf, ne, n_patch;
  int32_t tri_off;      // into tri   (3 int32 per face, body-local vertex ids)
  int32_t edge_off;     // into edge  (int4 a, b, c, d per edge; d = -1 on a boundary edge)
  int32_t v2f_ptr_off;  // into v2f_ptr (nv + 1 entries, relative to v2f_idx_off)
  int32_t v2f_idx_off;  // into v2f_idx (body-local face ids)
  int32_t patch_off;    // into patch headers
  int32_t mface_off;    // into mface (faces in marker-patch order)
  int32_t pad[2];
};

// One force-kernel block works on a "patch": a contiguous range of a
// topology's vertices (own vertices) plus the halo vertices that the
// elements touching them reference.
struct PatchHdr {
  int32_t own0, n_own, n_loc, loc_off;       // own range, local vertex count, loc_vert offset
  int32_t n_edge, edge_off, n_face, face_off;
  int32_t csr_off, slot_off, n_slot, pad;    // csr_ptr offset (n_own + 1), csr_slot offset
};

// element records local to a patch: local vertex indices (0xFFFF = none)
struct PEdge {
  uint16_t l[4];       // a, b (edge), c, d (wings)
  int32_t eid;         // body-local edge id; bit 31 set when this patch owns the edge
};
struct PFace {
  uint16_t l[3];
  uint16_t owned;      // 1 when this patch owns the face (energy bookkeeping)
  int32_t fid;         // body-local face id
};

// The force kernel's own packed copy of a patch's element records, moved into
// shared memory with one bulk copy (16-byte aligned, whole 16-byte units):
// 4 words per edge, 2 per face (each face attached to an edge of its own),
// then the first contribution slot of every own vertex (16 bits); its rest data
// (per work item: rest lengths, cos and sin of the rest angles, rest face
// areas, and the element multipliers of a varied body, in the patch's edge and
// face order) with a second one.
struct FPatch {
  int32_t blob_off;      // word offset in fblob (a multiple of 4)
  int32_t blob_words;    // 4 n_edge + 2 n_face + (n_own + 2) / 2, rounded up to a multiple of 4
  int32_t n_slot;        // contributions to the own vertices (one per edge role)
  int32_t vf_words;      // words after the blob read by the adjoint only: every own
                         //  vertex's first entry (n_own + 1 16-bit values), then its
                         //  faces as face | corner << 30, rounded up to a multiple of 4
};
__host__ __device__ constexpr int pad4(int n) { return (n + 3) & ~3; }
// rest words of a work item: l0, cos0, sin0 (pad4(n_edge) each), A0f
// (pad4(n_face)); a varied body adds kse, kbe and kaf
__host__ __device__ constexpr int frest_words(int n_edge, int n_face, bool varied) {
  return (varied ? 5 : 3) * pad4(n_edge) + (varied ? 2 : 1) * pad4(n_face);
}

struct Grid {
  int32_t n[3];
  float h[3], invh[3];
};

// scalars of one call
struct StepConsts {
  float dt, inv_dt, mu, probe_h;
  float kappa;           // 1 / (1.5 alpha)^2: W = exp(-kappa * (delta in cells)^2) per direction
  float cl_scale;        // (hx + hy + hz) / 3 / (hx hy hz): c_l = A_l * cl_scale
  int32_t forward_euler;
  int32_t starve_tx;     // bytes announced to the bulk-copy barriers beyond the copies: 0 in
                         //  use; the environment variable IBM_TEST_STARVE_TX sets it at
                         //  context creation, to test that every such wait runs out and
                         //  reports ERR_TIMEOUT
};

constexpr int kMT = 256;             // most markers (faces) per block of the marker kernel (a
                                     //  patch); the context picks 128 or 256 (marker_patch)

// ---------------------------------------------------------------------------
// tile-owned spread: the grid is cut into tiles of kTX x kTY x kTZ nodes (the
// last tile of a direction may be partial); each marker is listed under every
// tile that the union of its three components' 3x3x3 centroid supports
// reaches (nodes f-1 .. f+2 per direction, f = floor of the centroid in
// cells), and one block per tile sums what its nodes receive
// ---------------------------------------------------------------------------
constexpr int kTX = 16, kTY = 8, kTZ = 8;
constexpr int kTileNodes = kTX * kTY * kTZ;   // 1024 nodes, 128 x-segments of 8 nodes
constexpr int kTileThreads = 256;
// TileDev::state slots
enum : int32_t { TS_EPOCH = 0, TS_LEN = 1, TS_PAIRS = 2 };

struct TileDev {
  int32_t nt[3] = {0, 0, 0};    // tiles per direction
  int32_t n_tiles = 0;
  int32_t* count = nullptr;     // [n_tiles] markers reaching the tile in this call (the
                                //  spread kernel resets it to 0)
  uint32_t* tmax = nullptr;     // [n_tiles][4] largest |c_l F| per component of those
                                //  markers, as float bits (reset by the spread kernel)
  int32_t* off = nullptr;       // [n_tiles] first slot of the tile's markers in mlist
  int32_t* cur = nullptr;       // [n_tiles] fill cursor; after the fill, the end of the list
  int32_t* epoch = nullptr;     // [n_tiles] last clear-mode call in which markers reached it
  uint32_t* mask = nullptr;     // [n_tiles][3][4] x-segments of 8 nodes that the last
                                //  clear-mode spread left nonzero, per component
  int32_t* active[1] = {nullptr};  // [n_tiles] tiles listed in this call
  int32_t* state = nullptr;     // [8] TS_* counters
  int32_t* mlist = nullptr;     // [max_pairs] marker ids grouped by tile
  float4* rec = nullptr;        // [F][2] per marker: (centroid in cells relative to the body's
                                //  cell G, body id as bits, or -1 when not spread), (c_l F, 0)
};

// wrapped index of x into [0, n), any int x (one compare and add in the
// usual case of x within one period of the box)
__device__ __forceinline__ int wrap_any(int x, int n) {
  if (x >= 0 && x < n) return x;
  if (x < 0 && x >= -n) return x + n;
  if (x >= n && x < 2 * n) return x - n;
  x %= n;
  return x < 0 ? x + n : x;
}

// distinct tiles (at most 3) of direction d holding the nodes f - 1 .. f + 2
__device__ __forceinline__ int tiles_along(int f, int n, int T, int (&out)[3]) {
  int k = 0;
#pragma unroll
  for (int s = -1; s <= 2; ++s) {
    const int t = wrap_any(f + s, n) / T;
    bool dup = false;
#pragma unroll
    for (int j = 0; j < 3; ++j) dup = dup || (j < k && out[j] == t);
    if (!dup && k < 3) out[k++] = t;
  }
  return k;
}
constexpr int kForceThreads = 256;   // threads per force-kernel block
// host mirror of the node update's outputs (ibm_step_host): the force kernel
// writes x', v' to device arrays and the last block to complete each chunk of
// kMirrorChunk entries of the flat [3][V] arrays copies that chunk into host
// memory in whole lines
constexpr int kMirrorChunk = 2048;
struct Mirror {
  float* hx = nullptr;   // host x' and v' ([3][V]); null: no mirror
  float* hv = nullptr;
  int* count = nullptr;  // [ceil(3V / kMirrorChunk)] entries written per chunk (zeroed before)
  int vec = 0;           // both host arrays 16-byte aligned
};
constexpr uint16_t kNone = 0xFFFF;

// error word bits (device)
enum : int32_t { ERR_NONFINITE = 1, ERR_BAD_INDEX = 2, ERR_TILE_DENSE = 4, ERR_TIMEOUT = 8 };

struct DeviceTables {
  BodyDev* body = nullptr;
  TopoDev* topo = nullptr;
  int32_t* tri = nullptr;
  int4* edge = nullptr;
  int32_t* v2f_ptr = nullptr;
  int32_t* v2f_idx = nullptr;
  PatchHdr* patch = nullptr;
  int32_t* loc_vert = nullptr;
  PEdge* pedge = nullptr;
  PFace* pface = nullptr;
  int32_t* csr_ptr = nullptr;
  uint16_t* csr_slot = nullptr;
  uint32_t* fblob = nullptr;    // force-kernel element blobs (FPatch)
  FPatch* fpatch = nullptr;     // per topology patch, indexed like `patch`
  float* frest = nullptr;       // rest data of every work item, in patch order
  int64_t* wrest = nullptr;     // [n_work] word offset of the work item's rest data
  float* l0 = nullptr;          // [E] rest edge lengths
  float2* cs0 = nullptr;        // [E] (cos theta0, sin theta0) per hinge edge
  float* A0f = nullptr;         // [F] rest face areas
  float* kse = nullptr;         // [E] multiplier of k_s per edge (van Gelder / materials),
  float* kbe = nullptr;         // [E] of k_b per hinge edge, [F] of k_a per face;
  float* kaf = nullptr;         //     null when every body is uniform
  uint8_t* clamp = nullptr;     // [V]
  float* rest = nullptr;        // [3][V] body-frame rest positions
  int4* chunks = nullptr;       // (body, offset in the topology's mface list, count,
                                //  chunk index in body): one marker patch each
  int2* work = nullptr;         // (body, patch index within topology)
  unsigned long long* qsum = nullptr;  // [B][2] fixed-point (A, V) sums of the marker kernel:
                                       // one of two buffers, alternating between steps
  double* meas = nullptr;       // [B][2] (A, V) (formed from qsum by the finalize kernel)
  float2* coef = nullptr;       // [B] (k_A (A - A0)/A0, k_v (V - V0)/V0) (likewise)
  float* fext = nullptr;        // [3][F] scratch marker traction (ibm_step)
  int32_t* mface = nullptr;     // faces of every topology in marker-patch order (body-local)
  int4* mtri = nullptr;         // the same faces as (vertex a, b, c, face), body-local
  int4* boxes = nullptr;        // [n_chunks][2] footprint of each marker block's last spread:
                                // (x, y, z lo, kind: 0 rows, 1 whole box, 2 rows in float4
                                // groups), (x, y, z size, rows)
  int2* rowmap = nullptr;       // [n_chunks][kMaxRows] (global offset of the (y, z) row,
                                //  first x wrapped | length << 16): the x-range of each
                                //  footprint row that received a nonzero spread
  int32_t* stats = nullptr;     // [4] counters: marker blocks that did not fit shared memory
  // adjoint scratch
  double* partial2 = nullptr;   // [n_chunks][2] per-chunk (grad A . g, grad V . g)
  int32_t* counter2 = nullptr;  // [B]
  double* dmeas = nullptr;      // [B][2] per-body (grad A . g, grad V . g)
  float* gxe = nullptr;         // [9][F] per-face position cotangents (3 corners x 3)
  double* wpart = nullptr;      // [n_work][3] per-patch (g k_s, g k_b, g k_a)
  int32_t* wcounter = nullptr;  // [B]
  double* tpart = nullptr;      // [n_chunks][10] per-chunk volume moments
  double* taylor = nullptr;     // [B][24] moments, eigenvalues, extreme eigenvectors, gap
  double* tgrad = nullptr;      // [B][10] cotangents of the moments
  int32_t* err = nullptr;       // device error word
};

// marker-kernel dynamic shared memory: row tables (5 int arrays of kMaxRows;
// per staged float4 group its global offset and its row id), then two
// staging buffers of kMaxNodes words (velocity components, double-buffered;
// then the fixed-point spread accumulators of two force components)
constexpr int kMaxRows = 4 * kMT;                                  // (y, z) rows per patch
constexpr int kMaxNodes = 35 * kMT;                                // staged nodes per buffer
// (the staged-row-start array has kMaxRows + 4 entries, so every array
// starts on a 16-byte boundary)
constexpr int kRowTableBytes =
    ((4 * (5 * kMaxRows + 4) + 4 * (kMaxNodes / 4) + 2 * (kMaxNodes / 4)) + 15) / 16 * 16;
// Per-chunk cache of the coupled forcing launch (the markers stay at x^n for
// the three substeps of a coupled step): a 16-word header (x, y, z lo, x, y,
// z size, staged nodes, fits), then three row arrays (kMaxRows words each:
// staged offset - x0, row length, staged start), the groups' global offsets
// (kMaxNodes / 4 words) and their row ids (kMaxNodes / 4 16-bit ids)
constexpr int kCacheWords = 16 + 3 * kMaxRows + kMaxNodes / 4 + kMaxNodes / 8;
constexpr int kMarkerSmemBytes = kRowTableBytes + 8 * kMaxNodes;
// the same sizes for a marker patch of MT faces (kMaxRows, kMaxNodes and the
// cache layout are those of the largest patch, kMT)
__host__ __device__ constexpr int marker_rows(int MT) { return 4 * MT; }
__host__ __device__ constexpr int marker_nodes(int MT) { return 35 * MT; }
__host__ __device__ constexpr int marker_row_table_bytes(int MT) {
  return ((4 * (5 * marker_rows(MT) + 4) + 6 * (marker_nodes(MT) / 4)) + 15) / 16 * 16;
}
__host__ __device__ constexpr int marker_smem_bytes(int MT) {
  return marker_row_table_bytes(MT) + 8 * marker_nodes(MT);
}
static_assert(marker_smem_bytes(kMT) == kMarkerSmemBytes, "marker layout");

// elementwise combinations of [3][V] arrays for the strong-coupling integrator
constexpr int kLinCombMax = 6;
struct LinComb {              // out = sum_j c[j] in[j], j < k
  const float* in[kLinCombMax];
  float c[kLinCombMax];
  int k;
};
struct HamPredict {           // predictor p and modified value m (x and v parts)
  const float *x3, *v3, *vn, *vn1, *vn2, *an, *an1, *an2, *pcx, *pcv;
  float *px, *pv, *mx, *mv;
  float h;
  int first;                  // no p_n - c_n yet: m = p
};
struct HamCorrect {           // corrector, final value and p - c
  const float *xn, *vn, *x2, *v2, *vn1, *an, *an1, *mv, *am, *px, *pv;
  const uint8_t* clamp;
  float *xo, *vo, *pcx, *pcv;
  float h;
};

// 64-bit integer to float without a 64-bit conversion instruction
__device__ __forceinline__ float i64_to_float(long long d) {
  return fmaf((float)(int)(d >> 32), 4294967296.f, (float)(unsigned)(d & 0xffffffffll));
}

// global-term coefficients k_A (A - A0)/A0 and k_v (V - V0)/V0 from the
// fixed-point sums; the difference to the rest value is exact
__device__ __forceinline__ float2 body_coef(const BodyDev& B, unsigned long long qa,
                                            unsigned long long qv) {
  const float cA = i64_to_float((long long)qa - B.qA0) * B.cA_unit;
  const float cV = B.closed ? i64_to_float((long long)qv - B.qV0) * B.cV_unit : 0.f;
  return make_float2(cA, cV);
}

}  // namespace ibm

struct ibm_ctx {
  int device = 0;
  int marker_patch = ibm::kMT;      // faces per marker-kernel block: 128 or 256
  // coupled forcing (allocated by the first ibm_flow_step with this context):
  // the per-chunk tables and per-face geometry of substep 0, and the forcing's
  // own footprint record for the clears between substeps
  int32_t* fc_tab = nullptr;        // [n_chunks][kCacheWords]
  float4* fc_face = nullptr;        // [n_chunks][kMT][2] (centroid in cells, area), (V^b, ok)
  int4* fc_boxes = nullptr;         // [n_chunks][2]
  int2* fc_rowmap = nullptr;        // [n_chunks][kMaxRows]
  int spread_variant = 1;       // 1: spread inside the marker kernel (patch-owned, atomic
                                //  flush); 2: tile-owned spread kernels
  ibm::TileDev td;
  int64_t max_pairs = 0;
  float phi_bound = 1.f;        // bound on |phi| of the MLS shape functions (fixed-point scales)
  int tile_grid = 0;            // blocks of the persistent tile kernels
  cudaStream_t side = nullptr;  // second stream of ibm_step (spread beside the force kernel)
  // ibm_step_host: device copies of host-resident state (x, v in; x', v' out
  // when the caller's memory is not device-accessible), the stream that
  // copies the inputs in beside the footprint clear, and its events; made by
  // the first call
  float* hs_buf[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaStream_t hcopy = nullptr;
  cudaEvent_t ev_hfork = nullptr, ev_hcopy = nullptr;
  int* hs_count = nullptr;      // the host mirror's per-chunk counters
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaStream_t stream = nullptr;
  std::string err;
  int64_t V = 0, F = 0, E = 0, B = 0;
  int32_t n_topo = 0, n_chunks = 0, n_work = 0;
  int vec4 = 0;                 // nx % 4 == 0: float4 row access allowed
  ibm_params prm{};
  ibm_grid_desc gdesc{};
  ibm::Grid grid{};
  ibm::StepConsts sc{};
  size_t force_smem = 0;
  size_t adjoint_smem = 0;
  int32_t max_own = 0;
  bool have_prev = false;
  // the body sums alternate between two buffers from one ibm_step to the next,
  // so that a step's clear may zero its buffer while the previous step's force
  // kernel still reads the other (overlap inside captured multi-step graphs)
  unsigned long long* qsum_base = nullptr;   // [2][B][2]
  int qpar = 0;
  // strong coupling (Hamming predictor-corrector): history and scratch, each
  // array [3][V], allocated on the first ibm_step_pc
  struct PCState {
    int steps = 0;              // steps since ibm_pc_reset; the first three are Runge-Kutta
    bool have_pc = false;       // p_n - c_n of the previous step is available
    float* yx[3] = {};          // x of y_{n-1}, y_{n-2}, y_{n-3}
    float* yv[3] = {};          // v of the same
    float* a[3] = {};           // a_n, a_{n-1}, a_{n-2}
    float *pcx = nullptr, *pcv = nullptr, *px = nullptr, *pv = nullptr, *mx = nullptr,
          *mv = nullptr, *am = nullptr;
    float *sx = nullptr, *v2 = nullptr, *v3 = nullptr, *v4 = nullptr, *a2 = nullptr,
          *a3 = nullptr, *a4 = nullptr;   // Runge-Kutta stages
  } pc;
  bool timing = false;          // record phase events in ibm_step
  bool timed = false;           // a timed step has been recorded
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  std::vector<ibm::BodyDev> h_body;
  std::vector<void*> allocations;
  ibm::DeviceTables d;
};

namespace ibm {
// kernel launchers (defined in the kernel translation units)
// p, accel: optional cell-centred pressure and vertex accelerations (probe
// pressure with the marker-acceleration correction); after_clear: the launch
// directly follows launch_clear on the stream and may overlap it
cudaError_t launch_mls(ibm_ctx* c, const float* x, const float* v, const float* u,
                       const float* vv, const float* w, const float* p, const float* accel,
                       float* U, float* Fm, const float* Fm_in, float* Fext, float* fx, float* fy,
                       float* fz, bool measure, bool interp, bool probe, bool spread,
                       bool record_cells, bool after_clear = false);
cudaError_t launch_clear(ibm_ctx* c, float* fx, float* fy, float* fz);
cudaError_t launch_forcing(ibm_ctx* c, int substep, const float* x, const float* xv,
                           const float* u, const float* vv, const float* w, float* fx, float* fy,
                           float* fz);

// marker kernel without the spread, writing the spread records and counting
// the marker-tile pairs of the tile-owned spread (`accumulate`: into the
// fields' existing values, outside the clear-mode bookkeeping)
cudaError_t launch_mls_records(ibm_ctx* c, const float* x, const float* v, const float* u,
                               const float* vv, const float* w, const float* p,
                               const float* accel, const float* Fm_in, float* Fext, bool measure,
                               bool probe, bool accumulate);
// tile-owned spread (k_tile.cu): begin a call (epoch, list lengths, body
// sums), offsets of the tiles' lists, fill, and the spread itself
cudaError_t launch_tile_begin(ibm_ctx* c, bool accumulate, bool zero_sums);
cudaError_t launch_tile_spread(ibm_ctx* c, float* fx, float* fy, float* fz, bool accumulate);
cudaError_t tile_spread_occupancy(int* blocks_per_sm);
// zero the fixed-point body sums (before a measuring marker launch that does
// not follow a clear), and form meas / coef from them (after it)
cudaError_t zero_body_sums(ibm_ctx* c);
cudaError_t launch_measure_finalize(ibm_ctx* c);
cudaError_t launch_force(ibm_ctx* c, const float* x, const float* v, const float* Fext,
                         float* Fint, float* x_out, float* v_out, double* energy, bool advance,
                         const Mirror* mirror = nullptr);
cudaError_t launch_advance(ibm_ctx* c, const float* x, const float* v, const float* Fint,
                           const float* Fext, float* x_out, float* v_out);
// a = (F_int + F_ext^v)/m at x (zero on clamped nodes), from per-face F_ext
cudaError_t launch_accel(ibm_ctx* c, const float* x, const float* Fext, float* a);
cudaError_t launch_lincomb(ibm_ctx* c, float* out, const LinComb& L);
cudaError_t launch_ham_predict(ibm_ctx* c, const HamPredict& P);
cudaError_t launch_ham_correct(ibm_ctx* c, const HamCorrect& C);
cudaError_t launch_backward(ibm_ctx* c, const float* x, const float* v, const float* u,
                            const float* vv, const float* w, const float* p, const float* accel,
                            const float* gx_next, const float* gv_next, const float* gfx,
                            const float* gfy, const float* gfz, float* gx, float* gv,
                            double* gparams);
cudaError_t launch_taylor(ibm_ctx* c, const float* x, double* D);
// interpolation at the centroids and probe traction with the general MLS
// moment solve and the face geometry in float64 (k_mls64.cu)
cudaError_t launch_interp64(ibm_ctx* c, const float* x, const float* v, const float* u,
                            const float* vv, const float* w, float* U, float* Fm, float* Fext);
cudaError_t launch_taylor_backward(ibm_ctx* c, const float* x, const double* gD, float* gx);
cudaError_t set_force_smem_limit(size_t bytes);
cudaError_t set_adjoint_smem_limit(size_t bytes);
cudaError_t set_marker_smem_limit();
// message returned by ibm_last_error(NULL)
void set_global_error(const std::string& msg);
// the fluid phase (ibm_flow.cu): one RK3 predictor / projection on stream s,
// and the checks ibm_flow_step makes against a context
cudaError_t flow_predict(ibm_flow* fl, int l, float* u, float* v, float* w, const float* p,
                         cudaStream_t s);
cudaError_t flow_project(ibm_flow* fl, int l, float* u, float* v, float* w, float* p,
                         const float* fx, const float* fy, const float* fz, float fscale,
                         cudaStream_t s);
bool flow_matches(const ibm_flow* fl, const ibm_grid_desc& g, double dt, double mu);
cudaStream_t flow_stream(const ibm_flow* fl);
int flow_device(const ibm_flow* fl);
size_t flow_cells(const ibm_flow* fl);
// phase-timing events (no-ops unless timing is on)
cudaError_t flow_mark(ibm_flow* fl, int l, int k, cudaStream_t s);
cudaError_t flow_mark_struct(ibm_flow* fl, int k, cudaStream_t s);
}  // namespace ibm
