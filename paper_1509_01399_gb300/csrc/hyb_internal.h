// Internal declarations of the hybrid FEM/FDM library: launch arguments of
// the step kernels and the host-side launchers.  Not part of the C ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "hyb.h"

namespace hyb {

constexpr int kMaxSlots = 16;   // problems advanced by one step launch
constexpr int kStepBlock = 288;  // threads per block of the step kernel (9 warps)
constexpr int kTileX = 32;       // interior thread tile (x): one warp per tile row
constexpr int kTileY = 16;       // interior tile (y): two rows per consumer thread
constexpr int kBoxY = kTileY + 2, kHBoxY = kTileY + 1;

// x geometry of the interior tiles.  FP32 tiles start at x = 32 m (tile 0
// holds the face node x = 0, whose thread idles): with the row pitch a
// multiple of 8, a warp's 32 nodes are one aligned 128-byte segment and its
// stores fill whole 32-byte sectors (partly written sectors, shared by two
// blocks, cost L2 and DRAM work).  The box then starts 4 nodes left of the
// tile and is 40 wide.  FP64 tiles start at x = 1 + 32 m, the box at the
// halo node x = 32 m, 36 wide (256-byte rows; a 40-wide box would cost the
// second resident block).
template <typename T>
struct Box {
  static constexpr int x0 = sizeof(T) == 4 ? 0 : 1;    // first node of tile 0
  static constexpr int hx = sizeof(T) == 4 ? 4 : 1;    // box columns left of the tile
  static constexpr int BX = sizeof(T) == 4 ? 40 : 36;  // box width (a multiple of 16 bytes)
  static constexpr int C = BX * kBoxY;                 // u box
  static constexpr int H = BX * kHBoxY;                // edge-weight / stored-u box
  // u^{k-1} on tiles off the faces: only the tile's own nodes are read, so
  // the box has no y halo and (FP32) no x halo: PX x kTileY from x = i0 - phx
  static constexpr int phx = sizeof(T) == 4 ? 0 : 1;
  static constexpr int PX = sizeof(T) == 4 ? 32 : 34;
  static constexpr int P = PX * kTileY;
};
// first node (x) of interior tile 0 for a mesh of the given precision
inline int tile_x0(int precision) { return precision == HYB_FP32 ? Box<float>::x0 : Box<double>::x0; }
constexpr int kReduceBlocks = 512;
// The step kernels accumulate kGradPairScale times the voxel pairing of
// Eq. (gradient1) (integer edge weights 2 and 1 instead of 1/3 and 1/6).
constexpr double kGradPairScale = 6.0;
constexpr int kReduceThreads = 256;

// One problem (one source of one mesh) inside a step launch.
template <typename T>
struct Slot {
  const T* cur;      // forward: u^k        adjoint: lambda^{j+1}
  const T* prev;     // forward: u^{k-1}    adjoint: lambda^{j+2}
  T* next;           // forward: u^{k+1}    adjoint: lambda^j
  T* obs_w;          // forward: trace row k+1 (nullptr: not recorded)
  const T* obs_r;    // adjoint: cotangent row j
  T* hist_w;         // forward: FEM-owned box slot for u^{k+1} (or nullptr)
  const T* hist_r;   // adjoint: FEM-owned box slot holding u^j (or nullptr)
  int mask_f;        // absorbing faces of the step (forward: step k, adjoint: B_j)
  int mask_e;        // adjoint: absorbing faces of E_{j-1}
  int mask_c;        // adjoint: absorbing faces of C_{j+1}
  int src_mask;      // forward: faces carrying the plane-wave flux at step k (bits; 0: none)
  int obs_face;      // face recorded in the trace / receiving the cotangent
  // Plane wave of the slot's source: the flux term of node (i, j, k) on face f
  // is sf[f] p(t_k - h (d . ((i, j, k) - si0))), p(s) = sin(omega s) on [0, t1].
  double st;         // t_k
  double sf[6];      // tau^2 (2 / h) amp (-(d . n_f)) on the entry faces, 0 elsewhere
  double sd[3];      // unit direction d
  double sh;         // lattice spacing h
  int si0[3];        // entry corner (node index)
  double somega, st1;
  // paper-mode adjoint (forward rows on lambda): the cotangent row entering on
  // the observation face as inj_scale 2^b c_j, b the node's boundary axes
  const T* inj;
  T inj_scale;       // -tau / h^3
  const T* ccur;     // centre nodes of refined voxels, levels as cur/prev/next
  const T* cprev;
  T* cnext;
  T* chist_w;        // forward: centre values of u^{k+1} for the gradient (or nullptr)
  const T* chist_r;  // adjoint: centre values of u^j (or nullptr)
  int zf_cur, zf_prev;  // plane 0 of cur / prev in the field tensor map (tmf)
  int zf_hist;          // plane 0 of hist_r's box in the history tensor map (tmh)
  // the slot's coefficient: edge weights [3][wsz] (plane 0 of its x array in
  // the weight tensor map tmw) and the refined voxels' a; one set shared by
  // every slot, or one per slot for batches of independent problems
  const T* W;
  int zf_w;
  const T* avox;
};

// Lattice fields are stored with a row pitch px >= nx (a multiple of 8, so
// that rows start on 32-byte boundaries): node (i, j, k) of a field is
// element i + px (j + ny k).  The edge-weight box starts at an x origin wx0
// that is a multiple of 4 and has a row pitch wpx that is a multiple of 4;
// the FEM-owned box (history) at hx0, a multiple of 8, with a pitch hpx
// that is a multiple of 8.
template <typename T>
struct StepArgs {
  CUtensorMap tmf;   // field buffer (all levels and slots): {nx, ny, planes}, box Box<T>::BX x kBoxY x 1
  CUtensorMap tmw;   // edge weights: {wpx, wn1, 3 wn2}, box Box<T>::BX x kHBoxY x 1
  CUtensorMap tmh;   // history: {hpx, fn1, fn2 x boxes}, box Box<T>::BX x kHBoxY x 1
  CUtensorMap tmp;   // field buffer as tmf, box Box<T>::PX x kTileY x 1 (u^{k-1} off the faces)
  int* err;          // [0]: set when a pipeline wait timed out
  long long wait;    // cycles a pipeline wait may take (< 0: give up at once if not complete)
  int nx, ny, nz;
  int px;            // row pitch of lattice fields
  int fl[3], fh[3];  // FEM-owned node range (inclusive); fl[0] > fh[0]: no FEM
  int fn[3];         // FEM-owned box dims (history layout)
  int wl[3], wn[3];  // edge-weight box: nodes fl-1 .. fh+1
  int wx0, wpx;      // x origin and row pitch of the edge-weight arrays
  long long wsz;     // entries per axis array of the edge-weight box (wpx wn1 wn2)
  int hx0, hpx;      // x origin and row pitch of the FEM-owned (history) box
  const T* W;        // [3][wsz]: weight of the edge (p, p + e_axis) (of slot 0)
  double* G;         // FP64 gradient accumulator over unknown voxels (adjoint)
  int un[3];         // unknown voxel dims; voxel origins fl .. fl + un - 1
  T c2;              // tau^2 / h^2 (per-axis steps: tau^2 / dx_1^2)
  T r;               // (h - tau) / (h + tau), Eq. (eq:abs2)
  // per-axis steps dx_1, dx_2, dx_3 that differ (ani = 1; every level then
  // runs the per-axis kernels): kap[ax] = dx_1^2 / dx_ax^2 weighs the axis-ax
  // terms of the lattice rows and the edge weights, ra[ax] = (dx_ax - tau) /
  // (dx_ax + tau) is the absorbing coefficient of the faces normal to axis ax
  int ani;
  double kap[3];
  T kapt[3];         // kap in the field's precision
  T kdiag;           // -2 (kap[0] + kap[1] + kap[2]) in the field's precision: a lattice row's diagonal
  T ra[3];
  int npb;           // interior: tiles per plane of the interior box
  int ntx;           // interior: tiles along x
  const int* items;  // interior work items, one per block: (slot, tile, z0, z1)
  int nitems;
  int small;         // some axis has < 5 nodes: one generic kernel per level
  int nedge;         // edge tiles (128 nodes) per slot
  int nhe, nhr;      // step kernel: leading blocks of edge tiles, trailing blocks of refined rows
  int nslots;
  // refined region (nref == 0: nothing refined): unknown voxels bisected
  // once (12 tetrahedra around a centre node).  Trailing blocks of the step
  // launch evaluate the rows of their corners (the stencil row corrected by
  // the refined voxels around the node) and of their centres; the interior
  // blocks skip those nodes.
  int nref;                   // refined voxels (= centre nodes)
  int nrl;                    // corners of refined voxels (lattice rows of the refined region)
  const uint2* rpos;          // each such corner (i | j << 16, k)
  const unsigned char* rmask; // FEM-owned box: bit 0 = the node is a corner of a refined voxel,
                              // bit 1 = the voxel with its origin at the node is refined
  const int* rzr;             // per FEM-owned column (i - fl0) + fn0 (j - fl1): [kmin, kmax] of its
                              // refined corners (kmin > kmax: none)
  const int* rcid;            // per unknown voxel: its centre id if refined, else -1
  const T* avox;              // per unknown voxel: the coefficient a (of slot 0; slots carry their own)
  const unsigned char* refvox;// unknown voxels: 1 = refined
  const int* refvox_id;       // unknown id of each refined voxel (centre order)
  const uint2* rvxyz;         // its origin in unknown-voxel coordinates (x | y << 16, z)
  const double* k9;           // 9 x 9 stiffness of a refined unit voxel, a = 1 (level-0 pairing)
  // unit-voxel tables (a = 1, corners a + 2b + 4c, centre 8): K9 of the
  // refined voxel, dK[c][q] = K9[c][q] - K8[c][q] (q = 8: K9[c][8]) against
  // the Kuhn voxel, and the lumped masses of both
  T rK9[81];
  T rdK[72];
  T rm9[9], rm8[8];
  // fem_path HYB_FEM_TET_ALL: every interior node's row gathered over the Kuhn
  // tetrahedra of its voxels (the all-node kernels run every level)
  int tet;
  const double* acoef;        // a on the unknown voxels (1 on the other voxels)
  const double* kuhn;         // [6][4][4] element stiffness (unit spacing, a = 1), then [6] volumes
  const int* kuhn_v;          // [6][4] corner ids (a + 2b + 4c) of each tetrahedron's vertices
  // telegraph reading (HYB_MODEL_TELEGRAPH; nullptr: the wave model): per
  // FEM-owned node (history-box layout) s = tau D / (2 M), D the damping
  // lumped like the mass.  FEM rows then read
  // u^{k+1} = u^k + ((u^k - u^{k-1})(1 - s) + tau^2/h^2 lap) / (1 + s), the
  // forward's history keeps u^{k+1} - u^{k-1}, and the adjoint pairs it
  // with lambda^{k+1} weighted by the lumped mass shares (damp_sum).
  const T* sdamp;
  Slot<T> s[kMaxSlots];
};

// One time level of every slot: one launch of the step kernel (edge tiles,
// refined rows and interior blocks), or on lattices with fewer than 5 nodes
// on an axis one generic kernel over every node.
template <typename T>
int launch_forward_step(const StepArgs<T>& a, cudaStream_t st);
template <typename T>
int launch_adjoint_step(const StepArgs<T>& a, cudaStream_t st);
// Resident blocks per SM of the step kernel (for grid sizing), at least 1.
int step_blocks_per_sm(int precision, int adjoint);
// G[c] += voxel pairing of (u^0 in hist box, lambda^1) for one slot.
template <typename T>
void launch_pair(const StepArgs<T>& a, const T* hist, const T* lam, cudaStream_t st);
// Edge weights W from the per-voxel coefficient (and, if avox is set, the
// coefficient itself in the field precision); raises *flag when a value
// exceeds a_max or is not finite.
template <typename T>
void launch_set_coef(const StepArgs<T>& a, T* W, T* avox, const double* acoef, double a_max, int* flag,
                     cudaStream_t st);
// Telegraph reading: sdamp (history-box layout) from sigma on the unknown
// voxels, s_i = (tau / 2) sum over the voxels v around node i of
// sigma_v m_{v,i} (m = 1/4 on a voxel's diagonal corners, 1/12 on the
// others); raises *flag when a sigma is negative or not finite.
template <typename T>
void launch_set_damp(const StepArgs<T>& a, T* sdamp, const double* sigma, double dt, int* flag, cudaStream_t st);
// (The rows of the refined region, identical for the forward and the
// mass-scaled adjoint, and the adjoint's gradient pairing of refined voxels
// run in trailing blocks of the step kernel.)
// Gradient pairing of refined voxels for level 0 (u^0 from the history
// slots `hist`/`chist`, lambda^1 as the slots' cur/ccur).
template <typename T>
void launch_refined_pair(const StepArgs<T>& a, cudaStream_t st);
// Trace row of face f (c_p + n_p c_q order) from a lattice field.
template <typename T>
void launch_extract_face(const StepArgs<T>& a, const T* field, int f, T* row, cudaStream_t st);
// Copy the FEM-owned box of a lattice field into a history slot.
template <typename T>
void launch_extract_owned(const StepArgs<T>& a, const T* field, T* box, cudaStream_t st);

// ---- reductions and CG vector kernels (FP64) ----
// Misfit over [n_src][nsteps+1][stride]: partials of 1/2 w m (u-obs)^2 and
// (optionally) cot = w m (u - obs).
struct MisfitGeom {
  int n_src, nsteps, stride;
  int face[kMaxSlots];
  int np[kMaxSlots], nq[kMaxSlots];  // in-face extents (fast, slow)
  double wt;                         // time weight for k >= 1
  double hh[kMaxSlots];              // face weight scale per source (1, or the in-face cell area)
  int halve;                         // halve the face weight on the face border
};
template <typename T>
void launch_misfit(const MisfitGeom& g, const T* trace, const T* obs, T* cot, double* partials,
                   cudaStream_t st);
// out[0] = sum of `n` partials (one block, fixed order).
void launch_sum(const double* partials, int n, double* out, cudaStream_t st);
// g = scale * sum_s G_s + gamma * vol * (a - a0), G holding n_src arrays of n
void launch_grad_finalize(const double* G, int n_src, const double* a, double scale, double gamma,
                          double vol, double a0, double* g, long long n, cudaStream_t st);
// partials of: [0] sum g^2, [1] sum (a - a0)^2, [2] sum gp^2 with gp the
// projected gradient (g zeroed where a sits at a bound and g points out of
// [lo, hi]); kCgParts partial arrays of kReduceBlocks entries
constexpr int kCgParts = 3;
void launch_cg_norms(const double* g, const double* a, double a0, double lo, double hi, long long n,
                     double* partials, cudaStream_t st);
// d = -gp / vol + beta * d (beta = 0: d = -gp / vol), then the components of d
// that would leave [lo, hi] at once set to 0
void launch_cg_direction(const double* g, const double* a, double lo, double hi, double vol, double beta,
                         double* d, long long n, cudaStream_t st);
// partials of: [0] sum g d, [1] max |d|
void launch_cg_dir_stats(const double* g, const double* d, long long n, double* partials,
                         cudaStream_t st);
void launch_max(const double* partials, int n, double* out, cudaStream_t st);
// out = clip(a + alpha d, lo, hi); partials of sum (out - a0)^2
void launch_cg_axpy_clip(const double* a, const double* d, double alpha, double lo, double hi,
                         double a0, double* out, long long n, double* partials, cudaStream_t st);

// Allocation-free misfit (hyb_misfit_noalloc): block partials in a static
// device array.  noalloc_scratch() returns its device address on the current
// device; noalloc_max_entries() is the largest trace it accepts.
long long noalloc_max_entries();
cudaError_t noalloc_scratch(double** out);
template <typename T>
void launch_misfit_noalloc(const MisfitGeom& g, const T* trace, const T* obs, T* cot, double* scratch,
                           long long total, double* J_dev, cudaStream_t st);

}  // namespace hyb
