/*
 * hyb.h - C ABI of the GB300 hybrid FEM/FDM wave solver for conductivity
 * reconstruction (Beilina, arXiv 1509.01399).
 *
 * The library advances the hyperbolic model u_tt - div(a grad u) = 0 of
 * Model Problem 2 (Sec. 5, Eq. (model2)) on a box: a structured lattice of
 * nodes x = origin + h (i, j, k) on which the finite-difference leapfrog
 * Eq. (fdmschemeforward) runs, and a central finite-element block whose voxels
 * are cut into Kuhn tetrahedra and updated by the explicit lumped-mass scheme
 * Eq. (fem).  The two meshes overlap by one cell as in Algorithm 1: the FEM
 * block's boundary shell (omega_o) is owned by the FDM, the next shell inward
 * (omega_diamond) and everything inside it by the FEM.  Both schemes write one
 * shared field, so the copies of Algorithm 1 are identities.
 *
 * The unknown coefficient a is piecewise constant (Eq. (p0)), one value per
 * "unknown voxel": a cell of the FEM block whose eight corners are all
 * FEM-owned (cells fem_lo+1 .. fem_hi-2 on every axis).  a = 1 everywhere
 * else (Eq. (2.3)).  Unknown voxels are stored x fastest:
 *   a[(cz * uy + cy) * ux + cx],  (ux, uy, uz) = hyb_mesh_info.unknown_dims.
 *
 * Conventions common to every call:
 *  - Every array argument is a caller-owned DEVICE pointer unless stated.
 *    Field-typed arrays (trace, cotangent, observations, fields) are double
 *    for HYB_FP64 meshes and float for HYB_FP32 meshes; coefficient,
 *    gradient and CG arrays are always double.
 *  - Calls are asynchronous on the mesh's stream (hyb_set_stream).  Argument
 *    errors are returned synchronously; device-side failures surface at
 *    hyb_sync.  Every call returns a hyb_status and never throws or aborts.
 *    hyb_last_error() gives a message for the calling thread's last failure.
 *  - One mesh is used by one host thread at a time.
 *  - Faces are numbered f = 2 * axis + side: 0 = x-low, 1 = x-high,
 *    2 = y-low, 3 = y-high, 4 = z-low, 5 = z-high.
 *  - A trace row of face f lists its nodes with in-face coordinates (c_p, c_q),
 *    p < q the two other axes, at index c_p + n_p * c_q; rows are padded to
 *    hyb_mesh_info.obs_stride entries.
 */
#ifndef HYB_H_
#define HYB_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hyb_mesh hyb_mesh;

typedef enum {
  HYB_OK = 0,
  HYB_ERR_ARG = -1,     /* invalid argument (sizes, enums, null pointers) */
  HYB_ERR_CFL = -2,     /* dt above the stability bound, or a > a_max */
  HYB_ERR_OOM = -3,     /* device allocation failed */
  HYB_ERR_CUDA = -4,    /* a CUDA call failed */
  HYB_ERR_TIMEOUT = -5, /* a bounded device-side wait gave up */
  HYB_ERR_STATE = -6    /* call out of order (e.g. adjoint before forward) */
} hyb_status;

enum { HYB_BC_NEUMANN0 = 0, HYB_BC_ABC = 1 };
enum { HYB_FP64 = 0, HYB_FP32 = 1 };
enum { HYB_WEIGHTS_PLAIN = 0, HYB_WEIGHTS_QUADRATURE = 1 };
enum { HYB_FIELD_U_LAST = 0, HYB_FIELD_U_PREV = 1, HYB_FIELD_LAMBDA_FIRST = 2 };

/* Mesh description (Sec. 9 geometry; Algorithm 1 node classes). */
typedef struct {
  int32_t n[3];        /* lattice nodes per axis, each >= 3 */
  double h;            /* lattice spacing, the same on every axis (Eq. (CFL));
                          ignored when `spacing` is set */
  double origin[3];    /* world coordinates of node (0,0,0) */
  int32_t fem_lo[3];   /* FEM block node range, inclusive; fem_lo[0] < 0 = no */
  int32_t fem_hi[3];   /*   FEM block.  Needs 0 <= lo, hi <= n-1, hi - lo >= 2 */
  int32_t bc[6];       /* HYB_BC_* per face: d_n u = 0, or d_n u = -d_t u
                          discretised by Eq. (eq:abs2) */
  int32_t precision;   /* HYB_FP64, or HYB_FP32 (FP32 fields and stencils,
                          FP64 gradient accumulation and CG reductions) */
  int32_t ckpt_every;  /* 0: the forward keeps u on the FEM-owned nodes at
                          every level for the gradient; C > 0: it keeps full
                          fields every C steps and the adjoint recomputes each
                          segment */
  double a_max;        /* upper admissible bound of a (Eq. (admpar)); sets
                          dt_max = h / sqrt(3 a_max) (Eq. (CFL)) on unrefined
                          meshes */
  const uint8_t* refine_mask; /* HOST, one byte per unknown voxel (NULL: none):
                          non-zero marks a voxel refined once by bisection (the
                          local refinement of K_h, Sec. 7.1): its six Kuhn
                          tetrahedra are bisected along their refinement edge,
                          the voxel diagonal, at a new centre node.  Marked
                          voxels need every corner at least 2 nodes from the
                          outer faces. */
  int64_t wait_cycles; /* limit, in SM clock cycles, of each bounded wait of
                          the step kernels for their staged planes (0: the
                          default, 2^29 cycles, about 0.25 s).  A wait that
                          runs out makes the kernel stop and hyb_sync return
                          HYB_ERR_TIMEOUT; the field is then undefined.
                          HYB_WAIT_NONE (-1) gives up at the first wait that
                          is not already complete (error-path testing). */
  int32_t adjoint_mode; /* HYB_ADJ_EXACT: hyb_adjoint solves the exact
                          transpose of the discrete forward (its gradient is
                          the derivative of the discrete functional).
                          HYB_ADJ_PAPER: the paper's adjoint scheme,
                          Eq. (fdmschemeadjoint) and Eq. (fem) second line with
                          d_n lambda = 0 on every face (Eq. (adjoint1)), the
                          residual entering on S_T as the mirror ghost of
                          d_n lambda = -(u - u~), and the gradient
                          tau sum_k int grad u^k . grad lambda^k (Eq. (gradient1),
                          same time index).  With reflecting faces the two
                          agree; with absorbing faces they differ, because the
                          paper drops the absorbing terms of Eq. (lagrangian1). */
  int32_t fem_path;    /* HYB_FEM_STENCIL: the hybrid scheme; FEM rows on the
                          FEM block, in the exactly equal stencil form of the
                          Kuhn element matrices.  HYB_FEM_TET_ALL: pure FEM,
                          every interior lattice node updated by Eq. (fem) with
                          its row gathered element by element over the Kuhn
                          tetrahedra of every voxel (the coefficient still
                          given on the FEM block's unknown voxels, 1 elsewhere);
                          the outer boundary rows stay FDM.  A checking path
                          (slow, no refinement): on structured meshes the two
                          paths agree (the schemes coincide, Sec. 1, Sec. 7). */
  int32_t model;       /* HYB_MODEL_WAVE: u_tt = div(a grad u), the coefficient
                          arrays of the calls below are a.  HYB_MODEL_TELEGRAPH:
                          the damped reading u_tt + sigma u_t - div grad u = 0
                          (a = 1), the coefficient arrays are sigma >= 0 on the
                          unknown voxels (0 elsewhere); the damping is lumped
                          like the mass and central in time, so a FEM row reads
                          (1 + s) u^{k+1} = 2 u^k - (1 - s) u^{k-1} - tau^2 (M^L)^{-1} K u^k,
                          s_i = tau D_i / (2 M^L_i), and hyb_adjoint accumulates
                          dJ/dsigma_v = -tau/2 sum_k sum_i m_{v,i} lambda_i^{k+1} (u_i^{k+1} - u_i^{k-1})
                          (m_{v,i}: voxel v's lumped mass share of node i, in
                          units of h^3).  Needs a FEM block with fem_lo >= 2 and
                          fem_hi <= n - 3 on every axis, no refinement, the exact
                          adjoint and the stencil path, and no batches; a
                          negative sigma is reported by hyb_sync as HYB_ERR_CFL.
                          a_max keeps its role for the time step (a = 1). */
  double spacing[3];   /* lattice steps dx_1, dx_2, dx_3 per axis (the 7-point
                          Laplacian of Sec. 7.3 with unequal steps; the FEM
                          block's voxels are bricks, each cut into the six
                          Kuhn tetrahedra).  All 0: h on every axis.  Otherwise
                          each must be > 0 and h is ignored; equal steps are
                          the isotropic lattice.  Unequal steps: Eq. (eq:abs2)
                          takes r = (dx - tau) / (dx + tau) with dx the step
                          normal to each face (a node on several absorbing
                          faces: the mean of its per-face rows), the source
                          ghost 2 dx g uses that step too, the quadrature
                          weight of a face node is its in-face cell area
                          dx_p dx_q (halved on the face's border), and
                          dt_max = 1 / sqrt(a_max sum 1 / dx^2).  Every level
                          then takes two launches (the rows off the faces,
                          then the face layers by the generic rows; no staged
                          tiles).  Needs no refinement, the exact adjoint and
                          the wave model, and no batches (HYB_ERR_ARG). */
} hyb_mesh_desc;

#define HYB_WAIT_NONE (-1)
enum { HYB_ADJ_EXACT = 0, HYB_ADJ_PAPER = 1 };
enum { HYB_FEM_STENCIL = 0, HYB_FEM_TET_ALL = 1 };
enum { HYB_MODEL_WAVE = 0, HYB_MODEL_TELEGRAPH = 1 };

typedef struct {
  int64_t n_nodes;         /* lattice nodes */
  int64_t n_unknown;       /* unknown voxels */
  int64_t n_fem_owned;     /* FEM-owned nodes */
  int32_t unknown_dims[3];
  int32_t obs_stride;      /* padded length of one trace row */
  double dt_max;           /* stability bound for a <= a_max: h / sqrt(3 a_max)
                              (Eq. (CFL)), lowered by a row-sum bound of the
                              refined rows when voxels are refined; with
                              per-axis steps 1 / sqrt(a_max sum 1 / dx^2) */
  double voxel_volume;     /* h^3, or dx_1 dx_2 dx_3 */
  int64_t device_bytes;    /* device memory currently held by the mesh */
  int64_t launches;        /* kernels launched by this mesh so far */
  int64_t n_centres;       /* centre nodes of refined voxels */
  int64_t n_sparse_rows;   /* rows updated in sparse form (refined region) */
  int64_t n_sparse_nnz;    /* off-diagonal entries of those rows */
} hyb_mesh_info;

/* Plane-wave source of Eq. (f), p(s) = amp sin(omega s) for 0 <= s <= t1 =
   2 pi / omega and 0 otherwise.
   dir = (0, 0, 0): a face source, the Neumann flux d_n u = p(t) on `face`
   while t <= t1 (the S_{1,1} part of Eq. (model2)); after that the face
   takes the mesh's own condition.
   dir != 0: the plane wave u = F(t - d.(x - x0)), F' = p, travelling along
   d = dir / |dir| from the box corner x0 where d.x is smallest.  Every face
   whose outward normal n has d.n < 0 carries the flux
   d_n u = -(d.n) p(t - d.(x - x0)) until the pulse has crossed its farthest
   node (t <= t1 + max over the face of d.(x - x0)), then takes the mesh's own
   condition.  A face source is the case d = -n of its face.  (The paper
   launches its wave from one face; oblique incidence is this library's
   extension of Eq. (f).)
   `face` is the observation face S_T whose trace is recorded. */
typedef struct {
  int32_t face;
  double omega;
  double amp;
  double dir[3];
} hyb_source;

/* Create a mesh: node classes, FEM block, device workspaces.  `stream` is a
   cudaStream_t (NULL = the legacy default stream).  Errors: HYB_ERR_ARG for
   an invalid description, HYB_ERR_OOM, HYB_ERR_CUDA. */
hyb_status hyb_mesh_create(const hyb_mesh_desc* desc, void* stream, hyb_mesh** out);
hyb_status hyb_mesh_query(const hyb_mesh* mesh, hyb_mesh_info* out);
hyb_status hyb_mesh_destroy(hyb_mesh* mesh);
hyb_status hyb_set_stream(hyb_mesh* mesh, void* stream);

/* Forward solve, Algorithm 2 forward in time from u^0 = u^{-1} = 0
   (Model Problem 2; or from the state set by hyb_set_initial, Model
   Problem 1), one independent problem per source, all sources
   advanced by the same launches.
   a:      device double[n_unknown], the coefficient on the unknown voxels.
   src:    HOST array of n_src sources (1 <= n_src <= 16).
   nsteps: number of time steps N (u^1 .. u^N are computed).
   dt:     time step tau, 0 < dt <= dt_max (else HYB_ERR_CFL).
   trace:  device field[n_src][nsteps + 1][obs_stride]; row k receives u^k on
           the source's face (row 0 = u^0 = 0).
   The mesh keeps what the adjoint needs (coefficient, sources, time grid,
   the FEM-owned part of every level or the checkpoints).  An a value above
   a_max is reported by hyb_sync as HYB_ERR_CFL. */
hyb_status hyb_forward(hyb_mesh* mesh, const double* a, const hyb_source* src, int32_t n_src,
                       int32_t nsteps, double dt, void* trace);

/* Batched forward: n_src independent problems on the same lattice class
   advanced by the same launches, slot s with its own coefficient
   a + s * n_unknown (device double[n_src][n_unknown]) and source src[s];
   otherwise as hyb_forward.  hyb_adjoint then runs the batch's adjoints
   (cotangent [n_src][nsteps + 1][obs_stride], each slot accumulating its
   own gradient) and hyb_gradient_batch returns them one per slot.  This is
   the serving form's iteration-level batching (not a construct of the
   paper): a slot's arithmetic is the same alone and in a batch.  Not on the
   HYB_FEM_TET_ALL path. */
hyb_status hyb_forward_batch(hyb_mesh* mesh, const double* a, const hyb_source* src, int32_t n_src,
                             int32_t nsteps, double dt, void* trace);
/* Data misfit of every slot of the last forward on its own: J_host[s]
   (HOST double[n_src]; the call synchronises) = 1/2 sum_{k>=1, j} w_k m_j
   (u - u_obs)^2 over slot s's rows, as hyb_misfit computes it for a
   one-slot mesh; cotangent (device, may be NULL) as hyb_misfit. */
hyb_status hyb_misfit_batch(hyb_mesh* mesh, const void* trace, const void* u_obs, int32_t weights, double* J_host,
                            void* cotangent);
/* g_out[s] (device double[n_src][n_unknown]) = dJ_s/da_s + gamma |c| (a_s - a0)
   for every slot of the last batch (Eq. (gradient1) per problem). */
hyb_status hyb_gradient_batch(hyb_mesh* mesh, const double* a, double gamma, double a0, double* g_out);

/* Initial state of Model Problem 1 (Eq. (model1)): the forwards that follow
   start from u^0 = u0 and u^{-1} = u_prev instead of zero (Model Problem 2).
   u0, u_prev: device fields[n_nodes] of the mesh's precision (lattice nodes,
   x fastest), the same state for every source; c0, c_prev: device
   [n_centres] values on the centre nodes of refined voxels, in
   unknown-voxel order (NULL: zero).  The mesh copies them.  u0 == NULL
   returns to the zero state.  The gradient of a forward that started from
   a nonzero state pairs u^0 as well (the k = 0 term of Eq. (gradient1)). */
hyb_status hyb_set_initial(hyb_mesh* mesh, const void* u0, const void* u_prev, const void* c0,
                           const void* c_prev);

/* Exact discrete adjoint of the last hyb_forward, backward in time
   (the discrete counterpart of Eq. (adjoint1)): with c^k = dJ/d(trace row k)
   given in `cotangent` (device field[n_src][nsteps + 1][obs_stride]; row 0 is
   ignored), it solves the transposed time stepping from lambda^{N+1} =
   lambda^{N+2} = 0 and accumulates, in FP64,
       dJ/da_c = -tau^2 sum_{k=0}^{N-1} (lambda^{k+1})^T (M^L)^{-1} K_c u^k,
   the discrete form of int_0^T grad u . grad lambda dt (Eq. (gradient1)),
   summed over sources.  accumulate = 0 clears the accumulator first.
   Errors: HYB_ERR_STATE without a preceding forward. */
hyb_status hyb_adjoint(hyb_mesh* mesh, const void* cotangent, int32_t accumulate);

/* Gradient of the Tikhonov functional Eq. (functional) with respect to the
   unknown-voxel values (Euclidean, i.e. dF/da_c):
       g_out[c] = dJ/da_c + gamma |c| (a[c] - a0),
   dJ/da_c from the adjoint accumulator, |c| = h^3.  g_out: device
   double[n_unknown].  The accumulator is left unchanged. */
hyb_status hyb_gradient(hyb_mesh* mesh, const double* a, double gamma, double a0, double* g_out);

/* Data misfit part of Eq. (functional) for a trace recorded by the last
   forward's sources and time grid, against observations u_obs (both device
   fields shaped like the trace):
     J_data = 1/2 sum_{s, k>=1, j} w_k m_j (u - u_obs)^2
   with w_k = 1, m_j = 1 (HYB_WEIGHTS_PLAIN) or w_k = tau and m_j the lumped
   face weight h^2, halved on each border of the face
   (HYB_WEIGHTS_QUADRATURE).  If J_host != NULL the FP64 value is written
   there (host pointer; the call then synchronises the stream).  If
   cotangent != NULL it receives c = w m (u - u_obs), the input of
   hyb_adjoint.  Padding entries of each row are written as 0. */
hyb_status hyb_misfit(hyb_mesh* mesh, const void* trace, const void* u_obs, int32_t weights,
                      double* J_host, void* cotangent);

typedef struct {
  double gamma;      /* Tikhonov weight (Eq. (functional)) */
  double a0;         /* reference coefficient */
  double a_min;      /* admissible set [a_min, a_max] (Eq. (admpar)) */
  double a_max;
  int32_t weights;   /* HYB_WEIGHTS_* of the misfit */
} hyb_cg_params;

typedef struct {
  double* d;         /* device double[n_unknown], previous direction (caller-owned) */
  double gnorm2;     /* ||projected g^{m-1}||^2, 0 before the first iteration */
  double alpha;      /* previous step length, 0 before the first iteration */
  double J;          /* F(a^{m-1}), unused before the first iteration */
  int32_t iter;      /* m, 0 before the first iteration */
} hyb_cg_state;

typedef struct {
  double J;          /* F(a^m) */
  double J_data;
  double gnorm;      /* ||g^m||_{L2} over the unknown voxels (Step 3) */
  double gpnorm;     /* ||projected g^m||_{L2} (the norm in beta) */
  double alpha;      /* step taken */
  double beta;       /* Fletcher-Reeves beta^m */
  double dJ0;        /* directional derivative along d^m */
  double alpha_trial;
  double J_trial;
} hyb_cg_report;

/* One iteration of Algorithm 3 on the admissible set [a_min, a_max]
   (Eq. (admpar)): forward and adjoint at a^m (Step 1), the L2 gradient
   g^m = int grad u . grad lambda dt + gamma (a^m - a0), the Fletcher-Reeves
   direction d^m = -g^m + beta^m d^{m-1} (Step 2; d^0 = -g^0) of the projected
   gradient (components zeroed on voxels at a bound whose gradient points out
   of the set), with the components of d^m that would leave the set at once
   dropped and a restart d^m = -g^m when d^m is not a descent direction; a
   step length from a parabola through F(0), F'(0) and F at one trial step
   (the paper leaves this rule open: the trial step is 0.5 / max|d^m| at the
   first iteration and after a step that did not lower F, else the previous
   step length); the update a^{m+1} = clip(a^m + alpha d^m, a_min, a_max).
   a: device double[n_unknown], updated in place.  u_obs: device field shaped
   like the trace.  state, report: host structs.  Synchronises the stream
   twice (for the line search). */
hyb_status hyb_cg_step(hyb_mesh* mesh, double* a, const void* u_obs, const hyb_source* src,
                       int32_t n_src, int32_t nsteps, double dt, const hyb_cg_params* params,
                       hyb_cg_state* state, hyb_cg_report* report);

/* Copy a field of source `isrc` (HYB_FIELD_*: u^N or u^{N-1} of the last
   forward, the earliest adjoint level of the last adjoint) into `out`
   (device field[n_nodes], x fastest; lattice nodes only).  HYB_ADJ_EXACT:
   lambda^1, kept in the mass-scaled form lambda_i h^3 / M^L_i on FEM-owned
   rows, which equals lambda except at corners of refined voxels.
   HYB_ADJ_PAPER: lambda^0 of the paper's scheme.  On a checkpointing mesh the
   adjoint recomputes its segments in the forward's levels, so u^N and
   u^{N-1} are read before hyb_adjoint (HYB_ERR_STATE after it). */
hyb_status hyb_get_field(hyb_mesh* mesh, int32_t which, int32_t isrc, void* out);

/* Allocation-free data misfit.  The paper has no counterpart: this exists
   for callers that cannot allocate device memory when they need the misfit
   (code running while a stream is captured into a CUDA graph, loops where
   cudaMalloc's implicit device synchronisation is not allowed, hosts that
   serve all device memory from their own pool).  It computes what
   hyb_misfit computes, without a mesh: trace, u_obs (device fields of
   `precision`, shape [n_src][nsteps + 1][obs_stride]), face_dims (HOST
   int32[n_src][2]: the in-face extents (n_p, n_q) of each source's face),
   dt, h and `weights` as for hyb_misfit (one step h on every axis: the
   quadrature weight of a face node is h^2; meshes with per-axis steps use
   hyb_misfit).  Writes J_data to *J_dev (a DEVICE
   double) and, if cotangent != NULL, the cotangent, asynchronously on
   `stream` (a cudaStream_t; NULL = legacy default stream).
   It allocates nothing: its per-block partial sums live in a static
   128 KiB device array that every GPU loading the library holds until the
   process exits.  The trace may have at most 16384 * 4096 = 67,108,864
   entries (HYB_ERR_ARG beyond).  The first call on a device looks up that
   array's device address (cudaGetSymbolAddress) and caches it; make that
   first call before any stream capture.  All calls share the array, so calls
   that overlap on the GPU (different streams, or different host threads)
   race and must be serialised by the caller. */
hyb_status hyb_misfit_noalloc(const void* trace, const void* u_obs, int32_t precision, int32_t n_src,
                              int32_t nsteps, int32_t obs_stride, const int32_t* face_dims, double dt,
                              double h, int32_t weights, double* J_dev, void* cotangent, void* stream);

/* Wait for the mesh's stream, then report any device-side error flag:
   HYB_ERR_CFL for a coefficient above a_max (or not finite), HYB_ERR_TIMEOUT
   when a bounded wait of a step kernel ran out.  The flags are cleared. */
hyb_status hyb_sync(hyb_mesh* mesh);

/* Message of the calling thread's last failure ("" if none). */
const char* hyb_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* HYB_H_ */
