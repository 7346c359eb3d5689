/*
 * ibm.h -- C ABI of the GB300 Lagrangian hot path of the interaction-potential
 * + moving-least-squares immersed-boundary method (Spandan et al., "A parallel
 * interaction potential approach coupled with the immersed boundary method for
 * fully resolved simulations of deformable interfaces and membranes").
 *
 * One step, for many triangulated deformable bodies at once, with the Eulerian
 * velocity frozen:
 *   (a) internal nodal forces from the four interaction potentials (Sec. 2.3),
 *   (b) MLS interpolation of the staggered-grid velocity to the face-centroid
 *       markers, direct-forcing marker force and probe traction (Sec. 2.2),
 *   (c) node update m x'' = F_ext + F_int (Sec. 2.3; Sec. 5, step 4),
 *   (d) spreading of the marker forces back onto the grid (Sec. 2.2, Eq. mls_cl).
 *
 * Conventions (all entry points):
 *  - Every float* / double* argument except those marked "host" is a DEVICE
 *    pointer on the context's device, owned by the caller.  The context owns
 *    only topology, rest data and scratch.
 *  - Vertex arrays are float32 SoA [3][V]: x components first, then y, then z,
 *    vertices of body b at [v_off(b), v_off(b) + n_vert(b)) in body order.
 *    Positions are BODY-FRAME coordinates x - origin(b) (origin given per body
 *    at creation), which keeps edge vectors accurate in float32.
 *  - Per-face (per-marker) arrays are float32 SoA [3][F], faces in body order.
 *  - Eulerian fields are float32 [nz][ny][nx] (x fastest) on the MAC staggered
 *    lattice of the triply periodic box [0,L)^3: u at (i, j+1/2, k+1/2) h,
 *    v at (i+1/2, j, k+1/2) h, w at (i+1/2, j+1/2, k) h; force fields fx, fy,
 *    fz live on the u, v, w lattices respectively.
 *  - All calls are asynchronous and ordered on the context's stream (set with
 *    ibm_set_stream; default: the legacy default stream).  Only
 *    ibm_create_bodies and ibm_check_device_error synchronise.
 *  - Errors: a call returns an ibm_status; ibm_last_error() gives the message.
 *    No C++ exception crosses this interface.  Sizes are validated on the host.
 *  - The library never falls back to the CPU: without a usable CUDA device
 *    ibm_create_bodies returns IBM_ERR_CUDA.
 */
#ifndef IBM_GB300_H
#define IBM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ibm_ctx ibm_ctx;

typedef enum {
  IBM_OK = 0,
  IBM_ERR_INVALID_ARG = 1,  /* null pointer, bad size, bad parameter          */
  IBM_ERR_MESH = 2,         /* non-manifold / mis-oriented / degenerate mesh  */
  IBM_ERR_CUDA = 3,         /* CUDA runtime error (message has the details)   */
  IBM_ERR_DEVICE = 4,       /* device error word set by a kernel              */
  IBM_ERR_OOM = 5,          /* device allocation failed                       */
  IBM_ERR_UNSUPPORTED = 6   /* request outside the supported limits           */
} ibm_status;

/* One triangulated body (Sec. 2.2, Fig. lagmesh; the GTS-style vertex/face
 * lists of Sec. 5).  All pointers are HOST pointers, read during
 * ibm_create_bodies only.  Bodies whose (n_vert, tri) are identical share one
 * device copy of the topology tables. */
typedef struct {
  int32_t n_vert;
  int32_t n_face;
  const double* rest;      /* host [n_vert][3], absolute rest positions; the rest
                              state of every potential (l0, theta0, A0_f, A0, V0)  */
  const int32_t* tri;      /* host [n_face][3], counter-clockwise seen from the
                              outside (outward normals), 0-based vertex ids        */
  const uint8_t* clamped;  /* host [n_vert] or NULL; nonzero = node held fixed     */
  double origin[3];        /* body-frame origin (absolute), a point near the body  */
  double ks;               /* in-plane spring constant k_e (Eq. elaspot)           */
  double kb;               /* bending constant k_b                                 */
  double ka;               /* local area constant (per face, Eq. areapot)          */
  double kA;               /* global area constant (per body)                      */
  double kv;               /* volume constant (closed bodies; ignored if open)     */
  double mass;             /* node mass m (Sec. 2.3; 1 for drops)                  */
  int32_t closed;          /* 1 closed surface (one outward probe), 0 open sheet
                              (two probes, Sec. 2.2)                               */
  int32_t spring_model;    /* 0: k_e = ks on every edge; 1: van Gelder's model for
                              non-uniform meshes (Sec. 2.3), k_e = ks sum over the
                              edge's faces T of A_T / l_e^2 (rest values), ks then
                              being the membrane's E t                             */
  const float* face_material; /* host [n_face][3] or NULL: per-face multipliers of
                              (ks, kb, ka), >= 0 (e.g. two materials in one mesh);
                              an edge's spring takes the mean of its faces' (the
                              area-weighted sum under van Gelder), a hinge the mean
                              of its two faces', a face its own                    */
} ibm_body_desc;

typedef struct {
  int32_t n[3];            /* cells per direction (nx, ny, nz), each >= 4 */
  int32_t reserved;
  double L[3];             /* box lengths; h_d = L_d / n_d                */
} ibm_grid_desc;

typedef struct {
  double dt;               /* structural and forcing time step                   */
  double mu;               /* fluid viscosity in tau = mu (grad u + grad u^T)    */
  double alpha;            /* MLS weight shape parameter (Eq. mls_w); 0 -> 0.3   */
  double probe_h;          /* probe length; <= 0 -> mean grid spacing (Sec. 2.2) */
  int32_t theta0_zero;     /* 1: W_b = k_b(1 - cos theta) literally; 0: rest angle */
  int32_t forward_euler;   /* 1: forward Euler node update; 0: symplectic Euler  */
  int32_t patch_size;      /* vertices per force-kernel block; 0 -> default (128) */
  int32_t spread_variant;  /* how marker forces reach the grid (Eq. mls_cl):
                              1: inside the marker kernel, per marker patch, in
                                 exact fixed point, merged across patches with
                                 float atomics (order-dependent where patches
                                 meet; ibm_step clears the previous footprint
                                 with a separate kernel);
                              2: tile-owned: markers listed per 16x8x8-node tile,
                                 each tile's nodes summed in exact fixed point by
                                 one block and stored once with plain stores
                                 (bitwise deterministic; the previous step's
                                 footprint is zeroed in the same pass);
                              0: the library's default (1)                      */
  int32_t marker_patch;    /* faces per marker-kernel block (a surface patch of
                              one body): 128 or 256; 0 -> 256                   */
} ibm_params;

/* Create a context for n_bodies bodies on CUDA device `device`: validates the
 * meshes (Sec. 5 auxiliary arrays are built here: edges, faces of each edge,
 * the four vertices of each hinge, vertex->face incidence), computes the rest
 * state in float64 and uploads everything.  Synchronous.  On failure *out is
 * NULL and the status says why (IBM_ERR_MESH for bad meshes). */
ibm_status ibm_create_bodies(ibm_ctx** out, const ibm_body_desc* bodies, int32_t n_bodies,
                             const ibm_grid_desc* grid, const ibm_params* params,
                             int32_t device);

/* Free everything the context owns.  NULL is ignored. */
void ibm_destroy(ibm_ctx* ctx);

/* Message of the last failing call on ctx (or of the last failing
 * ibm_create_bodies when ctx is NULL).  Valid until the next call. */
const char* ibm_last_error(const ibm_ctx* ctx);

/* Stream (a cudaStream_t) on which all later calls are ordered. */
ibm_status ibm_set_stream(ibm_ctx* ctx, void* stream);

/* host out[6]: total vertices V, faces F, edges E, bodies B, distinct
 * topologies, force-kernel work items. */
ibm_status ibm_get_sizes(const ibm_ctx* ctx, int64_t* out);

/* host *out = the context's parameters as resolved at creation (defaults
 * filled in: patch_size, spread_variant, alpha, probe_h). */
ibm_status ibm_get_params(const ibm_ctx* ctx, ibm_params* out);

/* host out[3*B]: vertex, face, edge offset of every body. */
ibm_status ibm_get_offsets(const ibm_ctx* ctx, int64_t* out);

/* Initial state: x = rest - origin (float32, body frame), v = 0. */
ibm_status ibm_init_state(ibm_ctx* ctx, float* x, float* v);

/* Replace the elastic constants and masses: host consts[B][6] =
 * (ks, kb, ka, kA, kv, mass) per body.  Stream-ordered. */
ibm_status ibm_set_body_constants(ibm_ctx* ctx, const double* consts);

/* Per-body surface area A and enclosed volume V (Sec. 2.3: the global area
 * and volume of the potentials): out[B][2] float64 = (A, V); V is 0 for open
 * bodies.  Each face's float32 area (signed tetrahedron volume) is scaled by a
 * power of two chosen from the body's rest value, rounded to a 64-bit
 * integer and summed exactly, so the sums are independent of summation order
 * and carry a resolution of 2^-39 of the rest value (headroom 2^22). */
ibm_status ibm_body_measures(ibm_ctx* ctx, const float* x, double* out);

/* (a) Internal forces F_int = -grad(W_e + W_b + W_a + W_A + W_v) at x
 * (Sec. 2.3, Eqs. elaspot..areapot): F_int [3][V].  Deterministic: every
 * element's contribution is summed per vertex in a fixed order.  energy, if
 * not NULL: [B][5] float64 = (W_e, W_b, W_a local, W_A global, W_v). */
ibm_status ibm_compute_forces(ibm_ctx* ctx, const float* x, float* F_int, double* energy);

/* (b) MLS interpolation at the face centroids of the staggered velocity
 * (u, v, w) (Sec. 2.2, Eqs. mls..mls_Q), direct-forcing marker force
 * F = (V^b - U)/dt with V^b the mean velocity of the face's three nodes, and
 * probe traction F_ext = (-p n + tau . n) A (two probes on open sheets:
 * F_ext = (-(p+ - p-) n+ + (tau+ - tau-) . n+) A).
 * p: NULL (p = 0) or the pressure [nz][ny][nx] at the cell centres
 * ((i+1/2, j+1/2, k+1/2) h); the marker pressure is p* + h (Du/Dt).n with p*
 * interpolated at the probe end and Du/Dt the mean over the face's three
 * vertices of accel [3][V] (NULL: zero), each side of an open sheet with its
 * own normal.  Outputs [3][F], each may be NULL. */
ibm_status ibm_interpolate(ibm_ctx* ctx, const float* x, const float* v, const float* u,
                           const float* vv, const float* w, const float* p, const float* accel,
                           float* U, float* F_marker, float* F_ext);

/* The same as ibm_interpolate without pressure, with the MLS shape functions
 * of Eqs. mls_A..mls_Q from the general 4x4 moment system, factorised by LU
 * with partial pivoting, and the face geometry, both in float64 on the GPU
 * (the marker kernels use the exact closed form of the factorised weight in
 * float32).  It serves to measure the accuracy and the cost of that choice;
 * outputs are float32 [3][F], each may be NULL. */
ibm_status ibm_interpolate_fp64(ibm_ctx* ctx, const float* x, const float* v, const float* u,
                                const float* vv, const float* w, float* U, float* F_marker,
                                float* F_ext);

/* (c) Node update with F_ext^v = sum over faces of F_ext/3 (Sec. 2.3) and the
 * given F_int: symplectic (default) or forward Euler; clamped nodes keep x and
 * get v = 0.  x_out/v_out may alias x/v. */
ibm_status ibm_advance(ibm_ctx* ctx, const float* x, const float* v, const float* F_int,
                       const float* F_ext, float* x_out, float* v_out);

/* (d) Spread marker forces F_marker [3][F] at the centroids of x onto the
 * force fields: f_i^k += c_l phi_k^l F_i^l (Eq. mls_cl).  ACCUMULATES into the
 * caller's fields: with spread_variant 1 by atomic adds (summation order not
 * fixed), with 2 each touched node is read, added to and stored by one block
 * (deterministic). */
ibm_status ibm_spread(ibm_ctx* ctx, const float* x, const float* F_marker, float* fx, float* fy,
                      float* fz);

#define IBM_STEP_CLEAR_PREV 1u  /* zero the grid nodes the previous ibm_step of this
                                   context spread to, before spreading this step   */

/* One whole step (a)-(d) (three launches with spread_variant 1, six with 2):
 * x, v -> x_out, v_out (must not
 * alias x, v), spreading this step's marker forces into fx, fy, fz.  p and
 * accel as in ibm_interpolate (both may be NULL).  With
 * IBM_STEP_CLEAR_PREV the fields hold exactly this step's forces afterwards,
 * provided they held only the previous ibm_step's forces (or zeros) before. */
ibm_status ibm_step(ibm_ctx* ctx, const float* x, const float* v, const float* u,
                    const float* vv, const float* w, const float* p, const float* accel,
                    float* x_out, float* v_out, float* fx, float* fy, float* fz, uint32_t flags);

/* ibm_step with the body state in host memory: the same step, the same
 * results, but x, v, x_out, v_out ([3][V] float32) may be HOST arrays
 * (page-locked or ordinary) as well as device arrays; u, vv, w, p, accel and
 * the fields are device arrays as in ibm_step.  Host inputs are copied into
 * device arrays the context owns, on a second stream while the footprint
 * clear runs; outputs in device or page-locked host memory are written by
 * the force kernel directly (host memory over the host link), other host
 * outputs through the context's device arrays and a copy.  Synchronous:
 * returns when x_out, v_out hold the new state.  The first call allocates
 * the context's copies of the state (4 [3][V] float arrays), a stream and two
 * events.  Errors as ibm_step; like ibm_step it leaves the device error word
 * to ibm_check_device_error (after a kernel has flagged an error, x_out and
 * v_out may be incomplete). */
ibm_status ibm_step_host(ibm_ctx* ctx, const float* x, const float* v, const float* u,
                         const float* vv, const float* w, const float* p, const float* accel,
                         float* x_out, float* v_out, float* fx, float* fy, float* fz,
                         uint32_t flags);

/* Strong coupling (Sec. 2.3; the flow frozen, so the fluid-structure
 * iteration reduces to the structural integrator): one step of Hamming's
 * fourth-order predictor-corrector for y = (x, v), y' = (v, (F_int +
 * F_ext^v)/m): Milne predictor, Hamming modifier and corrector, final
 * correction, with two acceleration evaluations per step; the first three
 * steps after creation or ibm_pc_reset are classical Runge-Kutta steps (four
 * evaluations each).  Arguments, clamping, the spread of this step's marker
 * forces at (x, v) and the flags are as in ibm_step; p, accel may be NULL.
 * The context keeps the history (the three previous states and
 * accelerations), so each call's (x, v) must be the previous call's
 * (x_out, v_out); the first call allocates the history (about 24 [3][V]
 * float arrays), so make it before capturing a stream. */
ibm_status ibm_step_pc(ibm_ctx* ctx, const float* x, const float* v, const float* u,
                       const float* vv, const float* w, const float* p, const float* accel,
                       float* x_out, float* v_out, float* fx, float* fy, float* fz,
                       uint32_t flags);
/* Forget the predictor-corrector history: the next ibm_step_pc starts a new
 * trajectory with Runge-Kutta steps. */
ibm_status ibm_pc_reset(ibm_ctx* ctx);

/* Checkpoint and resume.  The context's own mutable state: the
 * strong-coupling history of ibm_step_pc (steps since ibm_pc_reset, the three
 * previous states, the two previous accelerations and the last
 * predictor-corrector difference; Sec. 2.3) and the record of the grid nodes
 * the last clear-mode step left nonzero in the caller's force fields (spread
 * variant 1: each marker patch's box and rows; variant 2: each tile's
 * clear-mode epoch and nonzero 8-node segments).  Positions, velocities,
 * fields and body constants belong to the caller and are not part of it.  A
 * context given the state of another context of the same bodies, grid, step
 * size and spread variant, with the caller's arrays as they were when it was
 * taken, continues exactly as the other would have: ibm_step_pc takes the same
 * predictor-corrector steps and a clear-mode step zeroes the same nodes.
 *
 * ibm_get_state: *size = the state's size in bytes; with buf != NULL the
 * state is also written to buf (HOST memory of `capacity` bytes; a smaller
 * capacity: IBM_ERR_INVALID_ARG, nothing written).  Synchronises the
 * context's stream and reports a device error word first (as
 * ibm_check_device_error), so no state is taken after a device error.
 *
 * ibm_set_state: reads `size` bytes of such a state from HOST memory buf;
 * IBM_ERR_INVALID_ARG (context unchanged) when it is truncated, was not
 * written by ibm_get_state of this format, belongs to a context of other
 * sizes, step size or spread variant, or holds a footprint record that names
 * nodes outside the grid.  Allocates the strong-coupling history if the state
 * holds one (so not inside a stream capture); synchronous. */
ibm_status ibm_get_state(ibm_ctx* ctx, void* buf, int64_t capacity, int64_t* size);
ibm_status ibm_set_state(ibm_ctx* ctx, const void* buf, int64_t size);

/* Adjoint of one step (a vector-Jacobian product, loose coupling with the
 * flow frozen; Sec. 2.3 node update, Sec. 2.2 traction and spreading, Sec. 2.3
 * potentials): given cotangents gx_next, gv_next [3][V] of the positions and
 * velocities an ibm_step from (x, v) produced, and optionally cotangents
 * gfx, gfy, gfz of the spread force fields [nz][ny][nx] (all three or none),
 * writes the cotangents gx, gv [3][V] of x and v and gparams [B][5] float64 =
 * cotangents of (k_s, k_b, k_a, k_A, k_v) per body.  The velocity field
 * (u, v, w) is the one the step used.  Included: the step's dependence on x
 * through the internal forces (exact Hessian-vector products of the four
 * potentials, including the per-body global area and volume terms), through
 * the probe traction (area, normal and the MLS velocity gradient at the probe
 * end, with its second derivatives) and, when the field cotangents are given,
 * through the spread f_i^k = c_l phi_k(c_l) (V^b_i - U_i(c_l))/dt (centroid,
 * area, and the vertex velocities in V^b; spreading transposed is MLS
 * interpolation weighted by c_l).  v may be NULL when the field cotangents are
 * (it enters only the spread).  p and accel are the ones the step used (NULL
 * allowed); the pressure load's dependence on x (area, normal, the MLS
 * pressure gradient at the probe ends) is included, accel is held fixed.
 * Outputs must not alias the cotangents.  Per-body sums are in a fixed order;
 * the result is deterministic.  Uses the context's per-face scratch (no
 * ibm_step may run concurrently on the context). */
ibm_status ibm_backward(ibm_ctx* ctx, const float* x, const float* v, const float* u,
                        const float* vv, const float* w, const float* p, const float* accel,
                        const float* gx_next, const float* gv_next, const float* gfx,
                        const float* gfy, const float* gfz, float* gx, float* gv,
                        double* gparams);

/* Taylor deformation D = (L - B)/(L + B) of every closed body (Sec. 3.1's
 * semi-axes L, B of a deformed drop), taken from the ellipsoid with the same
 * volume second moments: semi-axes sqrt(5 lambda_i) of the second-moment
 * tensor about the centroid, summed over signed tetrahedra in float64 in a
 * fixed order.  D [B] float64 (0 for open bodies). */
ibm_status ibm_taylor_deformation(ibm_ctx* ctx, const float* x, double* D);

/* Adjoint of ibm_taylor_deformation at x: given gD [B] float64, writes
 * gx [3][V] = d(sum_b gD_b D_b)/dx (overwritten, zero on open bodies) and D
 * [B] (recomputed at x).  Bodies whose largest and smallest eigenvalues
 * coincide (a sphere) have no derivative and get gx = 0. */
ibm_status ibm_taylor_backward(ibm_ctx* ctx, const float* x, const double* gD, float* gx,
                               double* D);

/* A CUDA graph of n_steps consecutive ibm_step calls (n_steps even, >= 2)
 * with the footprint clear: steps alternate (xa, va) -> (xb, vb) and back,
 * so after a launch the state is again in (xa, va).  The buffers and fields
 * are bound at creation; ibm_graph_launch replays the whole sequence on the
 * context's stream with one launch.  Inside the graph the force fields of the
 * intermediate steps are never observed, so each step's footprint clear runs
 * concurrently with the previous step's force kernel; after a launch fx, fy,
 * fz hold exactly the last step's forces.  As in ibm_step, each force kernel
 * may start while the marker kernel before it finishes (programmatic launch:
 * it waits for the marker kernel before using its results).  Creation
 * captures on a private stream after the work already queued on the
 * context's stream.  The context must outlive the graph. */
typedef struct ibm_graph ibm_graph;
ibm_status ibm_graph_create(ibm_ctx* ctx, float* xa, float* va, float* xb, float* vb,
                            const float* u, const float* vv, const float* w, const float* p,
                            const float* accel, float* fx, float* fy, float* fz, int32_t n_steps,
                            ibm_graph** out);
ibm_status ibm_graph_launch(ibm_graph* graph);
void ibm_graph_destroy(ibm_graph* graph);

/* Read a GTS (GNU Triangulated Surface) file, the format the paper's meshes
 * are exported in (Sec. 5): a header line "nv ne nf", nv lines "x y z", ne
 * lines of two 1-based vertex indices (edges), nf lines of three 1-based edge
 * indices (faces); blank lines and lines starting with '#' are skipped, and
 * anything after the numbers on a line is ignored.  A face's vertex order
 * follows its edges: the vertex of e1 not on e2, the vertex e1 and e2 share,
 * then the vertex of e2 not on e1 (so an oriented mesh stays oriented).
 * Two calls: with xyz and tri NULL it sets *n_vert and *n_face; then with
 * HOST buffers xyz[n_vert][3] (float64) and tri[n_face][3] (int32, 0-based)
 * and the sizes of the first call it fills them.  No context and no GPU are
 * needed.  Errors: IBM_ERR_INVALID_ARG (unreadable file, malformed line,
 * buffers not matching), IBM_ERR_MESH (index out of range, edges of a face
 * not forming a triangle); the message is in ibm_last_error(NULL). */
ibm_status ibm_gts_read(const char* path, int64_t* n_vert, int64_t* n_face, double* xyz,
                        int32_t* tri);

/* ---- The fluid phase and the coupled step (Sec. 2.1; Sec. 5 step 3) -------
 * Incompressible Navier-Stokes, Eqs. ns and con, density 1 and kinematic
 * viscosity nu = 1/Re, on the triply periodic MAC grid of the conventions
 * above, with the pressure at the cell centres (i+1/2, j+1/2, k+1/2) h.
 * Second-order centred conservative differences (divergence form) for the
 * nonlinear terms, 7-point Laplacians for the viscous terms, and the
 * self-starting three-substep RK3 fractional step: substep l = 0, 1, 2 with
 * gamma = (8/15, 5/12, 3/4), rho = (0, -17/60, -5/12), alpha = gamma + rho,
 *   (u* - u)/dt = gamma_l H(u) + rho_l H(u_prev) - alpha_l grad p
 *                 + alpha_l nu/2 lap(u* + u)                      (predictor)
 * with the implicit operator approximately factorised into
 * (1 - a d_xx)(1 - a d_yy)(1 - a d_zz), a = alpha_l dt nu/2, then
 *   lap(phi) = div(u*)/(alpha_l dt),  u = u* - alpha_l dt grad(phi),
 *   p <- p + phi - a lap(phi)                                      (projection).
 * In the periodic box both implicit operators are diagonal in Fourier space.
 * The Poisson equation is solved there (cuFFT transforms, float32).  The
 * factorised viscous operator is inverted exactly in one of two ways, fixed
 * per substep at creation: in real space when every direction's periodic
 * inverse, a circulant whose entries fall off as r^|m|, has less than 2^-26
 * of its mass beyond some |m| = W <= 8 with 2W + 1 <= n (then three
 * separable (2W+1)-tap filters, fused with the u* update; small
 * alpha_l dt nu / h^2), else in Fourier space.  A flow object owns its work
 * arrays (about thirteen fields) and FFT plans; velocity and pressure fields
 * are caller-owned device arrays [nz][ny][nx]. */
typedef struct ibm_flow ibm_flow;

/* Create a solver for grid (n >= 4 per direction; the reserved field is
 * ignored) with viscosity nu >= 0 and time step dt > 0, on the current
 * device; its calls run on the legacy default stream until
 * ibm_flow_set_stream.  Errors (message in ibm_last_error(NULL)):
 * IBM_ERR_INVALID_ARG, IBM_ERR_UNSUPPORTED (2^31 cells or more, n_z above
 * 65535 or n_y above 524280), IBM_ERR_OOM,
 * IBM_ERR_CUDA (no device, FFT plan). */
ibm_status ibm_flow_create(const ibm_grid_desc* grid, double nu, double dt, ibm_flow** out);
ibm_status ibm_flow_set_stream(ibm_flow* flow, void* stream);
/* The viscous solve of substep `substep` (0, 1, 2): *width = W >= 0 when it
 * runs in real space with 2W + 1 taps per direction, -1 when it runs in
 * Fourier space.  Host only.  Errors: IBM_ERR_INVALID_ARG. */
ibm_status ibm_flow_solve_width(const ibm_flow* flow, int32_t substep, int32_t* width);
/* Waits for the device to finish (coupled steps may still run on a
 * context's stream), then frees everything the flow owns.  NULL is ignored. */
void ibm_flow_destroy(ibm_flow* flow);

/* Predictor of RK3 substep `substep` (0, 1, 2): u, v, w <- u* in place, with
 * p the pressure of the previous substep.  The nonlinear terms H(u) are kept
 * in the flow object for the next substep's rho term, so the substeps of one
 * time step must run in order (substep 0 needs none). */
ibm_status ibm_flow_predict(ibm_flow* flow, int32_t substep, float* u, float* v, float* w,
                            const float* p);

/* Projection of substep `substep`: the provisional field u* + f_scale f
 * (fx, fy, fz on the u, v, w lattices; all three NULL: no forcing) is made
 * discretely solenoidal, u, v, w <- u; p is updated in place. */
ibm_status ibm_flow_project(ibm_flow* flow, int32_t substep, float* u, float* v, float* w,
                            float* p, const float* fx, const float* fy, const float* fz,
                            float f_scale);

/* One loosely coupled time step (Sec. 5 steps 1-4) on the context's stream:
 * three substeps of predictor, IBM forcing and projection, where the forcing
 * interpolates u* at the face centroids of x, forms F = (V^b - U*)/dt with
 * V^b the centroid velocity of xv, spreads it into fx, fy, fz (overwritten:
 * the last substep's forcing is left there) and adds dt f to u* (markers at
 * x throughout); then the bodies advance x, xv -> x_out, v_out as ibm_step
 * does, with the probe traction and pressure of the new u, v, w, p (no
 * acceleration correction).  ctx NULL: the flow alone (x ... fz may be
 * NULL).  The context's grid and dt must equal the flow's and its mu the
 * flow's nu (density 1); x_out, v_out must not alias x, xv.  Stability: with
 * the narrow MLS kernel a marker corrects its nearest node with a gain of
 * about A_l/h^2, so faces must stay below about two grid cells in area (the
 * paper's meshes keep triangles near the grid size); coarser meshes make the
 * slip, and then the flow, grow from substep to substep.  The first call with
 * a context allocates that context's forcing cache (per marker patch its
 * geometry and row tables, kept across the three substeps, and a footprint
 * record of its own, so ibm_step's clear is not disturbed): make it outside
 * a stream capture.  Errors:
 * IBM_ERR_INVALID_ARG on a mismatch or a null argument (message in
 * ibm_last_error(NULL) and, with a context, ibm_last_error(ctx));
 * IBM_ERR_OOM when the forcing cache cannot be allocated. */
ibm_status ibm_flow_step(ibm_flow* flow, ibm_ctx* ctx, const float* x, const float* xv,
                         float* x_out, float* v_out, float* u, float* v, float* w, float* p,
                         float* fx, float* fy, float* fz);

/* Phase timing of the flow (profiling aid, no counterpart in the paper):
 * when on, every predictor and projection records CUDA events around its
 * kernels and FFTs, and ibm_flow_step also around the body update.
 * ibm_flow_get_phase_times waits for the last recorded events and writes host
 * ms[13], each summed over substeps 0, 1, 2 of the last ones recorded:
 * (advection and right-hand side, forward FFT x3, Crank-Nicolson scaling,
 * inverse FFT x3 (these three 0 in real-space substeps), u* update (with the
 * real-space solve in it), IBM forcing (the time between predictor and
 * projection: force-field zeroing and the marker kernel), divergence,
 * forward FFT, Poisson scaling, inverse FFT, projection), then the body
 * update's marker kernel (body sums, probe traction) and force kernel
 * (0 when no coupled step was timed).  IBM_ERR_INVALID_ARG until each
 * substep has been timed once. */
ibm_status ibm_flow_set_phase_timing(ibm_flow* flow, int32_t on);
ibm_status ibm_flow_get_phase_times(ibm_flow* flow, float* ms);

/* Synchronise the stream and report the device error word (IBM_ERR_DEVICE if
 * a kernel flagged an out-of-range or non-finite value, too many markers in
 * one spread tile, or a wait for a bulk copy into shared memory that ran out:
 * every such wait is bounded (about a second), after which the block sets the
 * flag and returns; the word is reset by this call).  For testing that path,
 * the environment variable IBM_TEST_STARVE_TX (bytes, at most 1024), when set
 * at context creation, makes those waits expect more bytes than arrive. */
ibm_status ibm_check_device_error(ibm_ctx* ctx);

/* Phase timing of ibm_step (profiling aid, no counterpart in the paper): when
 * on (nonzero), every ibm_step records CUDA events on the context's stream
 * between its kernels.  ibm_get_phase_times waits for the last recorded step
 * and writes host ms[4] = (footprint clear (spread variant 1) or call set-up
 * (variant 2), marker kernel (with the spread in variant 1), tile-owned
 * spread (variant 2; 0 in variant 1), force+update kernel) of that step. */
ibm_status ibm_set_phase_timing(ibm_ctx* ctx, int32_t on);
ibm_status ibm_get_phase_times(ibm_ctx* ctx, float* ms);

/* Diagnostic counters since creation (synchronises): host out[4] =
 * (marker blocks whose stencil box did not fit shared memory and took the
 * direct global path, 0, 0, 0). */
ibm_status ibm_get_counters(ibm_ctx* ctx, int64_t* out);

/* Per-body surface area and enclosed volume WITHOUT a context and without
 * allocating any memory (no counterpart in the paper: it serves callers that
 * cannot allocate device memory at the point of the call, for example code
 * that runs inside another framework's memory pool or that must not add
 * allocations while a stream is being captured).  Each face's float32 area
 * and signed volume are summed in float64 in a fixed order (deterministic);
 * the result agrees with ibm_body_measures, which rounds each face to 2^-39
 * of the body's rest value before an exact integer sum, to about that
 * resolution.
 *   x         device float32 [3][n_vert], body-frame positions (SoA)
 *   tri       device int32 [F][3], GLOBAL vertex ids, faces of body b at
 *             [face_off[b], face_off[b+1]); F = face_off[n_bodies] faces
 *             must be readable
 *   face_off  device int32 [n_bodies + 1]
 *   max_faces_per_body  must bound face_off[b+1] - face_off[b] for every b
 *   closed    device uint8 [n_bodies] or NULL (all closed); open bodies get V = 0
 *   out       device float64 [n_bodies][2] = (A, V)
 *   stream    cudaStream_t (NULL: legacy default stream)
 * Scratch lives in one static device array of 1.25 MiB that every GPU
 * loading the library keeps until the process exits; limits: n_bodies <=
 * 65535 and n_bodies * ceil(max_faces_per_body / 256) <= 65536, larger
 * requests return IBM_ERR_UNSUPPORTED.  The first call on a device looks up
 * the array's device address (no allocation); make that first call before
 * any stream capture.  All calls share the array: calls that overlap on the
 * GPU (different streams, or different host threads) race and must be
 * serialised by the caller.  Device-side checks, made before any caller
 * index is used as an address: a body whose face range is negative or
 * reversed, has more faces than max_faces_per_body, or holds a vertex id
 * outside [0, n_vert) gets out = (NaN, NaN); a body with no faces gets (0, 0).
 * Errors: see ibm_last_error(NULL). */
ibm_status ibm_body_measures_noalloc(const float* x, int64_t n_vert, const int32_t* tri,
                                     const int32_t* face_off, int32_t n_bodies,
                                     int32_t max_faces_per_body, const uint8_t* closed,
                                     double* out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* IBM_GB300_H */
