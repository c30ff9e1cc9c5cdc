// Time-step kernels of the hybrid FEM/FDM scheme.
//
// One time level of every slot (source / problem) is one launch of
// step_kernel: its leading blocks run the edge tiles (nodes within one node
// of two faces), the next ones the interior (all other nodes), one work item
// (slot, 32 x 16 tile, z range) each, and its trailing blocks the rows of
// the refined region.  All
// blocks read levels k and k-1 and write disjoint nodes of level k+1.  An
// interior block's producer warp stages the planes it needs (u^k with a
// one-node halo, u^{k-1}, FEM edge weights, stored history) into shared
// memory with bulk tensor copies, one level ahead on items with FEM-owned
// nodes and six on the others (which stage only u^k and u^{k-1}); its
// eight consumer warps (two tile rows per thread) march the z range reading
// only shared memory, synchronised with the producer by per-level mbarriers
// only.  In tiles with one x face, lanes of the producer warp compute the
// column next to that face.  Consecutive launches overlap through
// programmatic dependent launch.
// Row kinds:
//  * FDM rows, Eq. (fdmschemeforward): u^{k+1} = 2u^k - u^{k-1} + tau^2 Delta_h u^k,
//  * FEM rows on the FEM-owned nodes, Eq. (fem) with lumped mass: on the
//    Kuhn-cut voxels the row is a 7-point stencil whose axis-edge weight is
//    W = sum over the four voxels around the edge of a_c / 3 (edge touching
//    the voxel's diagonal corners) or a_c / 6,
//  * boundary rows: Neumann mirror ghosts, the plane-wave flux of Eq. (f),
//    and the absorbing rows of Eq. (eq:abs2), which use the new value of the
//    inward neighbour: the thread of that neighbour writes the face node, and
//    edge/corner threads recompute the values they need, so no intra-step
//    synchronisation between blocks is needed.
// Both schemes write the same field, so the omega_o / omega_diamond copies
// of Algorithm 1 need no data movement.
//
// The transposed step is the exact transpose of the forward step (the
// discrete form of Eq. (adjoint1)).  Away from the outer boundary the
// mass-weighted operator is symmetric, so the transposed row is the forward
// stencil; next to a face the transposed face row (closed form) and its
// coupling are added, and near edges each node gathers the transposed
// coefficients of its neighbours' rows (mirror factors, absorbing rows) and
// solves the transposed absorbing coupling by recomputing the outer values.
// The same launch accumulates, per unknown voxel and in FP64, the sum over
// the voxel's 12 axis edges of w_e (u_p - u_q)(lambda_p - lambda_q) with
// w_e = 2 or 1 (six times the edge weights 1/3 and 1/6); the host scales it
// by -tau^2 / (6 h^2) (Eq. (gradient1)).
//
// Lattices whose steps differ per axis (the 7-point Laplacian of Sec. 7.3
// with dx_1, dx_2, dx_3) do not use step_kernel: each level is a bulk launch
// over the nodes off the faces (plain rows with per-axis weights) and a shell
// launch over the face layers (the generic rows), see ani_fwd_bulk_kernel.
#include "async_copy.cuh"
#include "hyb_internal.h"

namespace hyb {
namespace {

__device__ __forceinline__ int face_bits(int i, int j, int k, int nx, int ny, int nz) {
  return (i == 0 ? 1 : 0) | (i == nx - 1 ? 2 : 0) | (j == 0 ? 4 : 0) | (j == ny - 1 ? 8 : 0) |
         (k == 0 ? 16 : 0) | (k == nz - 1 ? 32 : 0);
}

// Plane-wave flux term tau^2 (2 / h) g of node (i, j, k) on flux face f
// (the mirror ghost u_g = u_in + 2 h g of d_n u = g, Eq. (f)):
// g = amp (-(d . n_f)) p(t_k - d . (x - x0)), p(s) = sin(omega s) on [0, t1]
// and 0 elsewhere.  The delay is formed in FP64; the pulse in the field's
// precision.
template <typename T>
__device__ __forceinline__ T src_term(const Slot<T>& S, int f, int i, int j, int k) {
  const double s =
      S.st - S.sh * (S.sd[0] * (i - S.si0[0]) + S.sd[1] * (j - S.si0[1]) + S.sd[2] * (k - S.si0[2]));
  if (!(s >= 0.0 && s <= S.st1)) return T(0);
  if constexpr (sizeof(T) == 4) return (T)S.sf[f] * sinf((float)(S.somega * s));
  else return (T)(S.sf[f] * sin(S.somega * s));
}

// Sum of the flux terms of the faces in `faces` (bits) that carry the flux.
template <typename T>
__device__ __forceinline__ T src_terms(const Slot<T>& S, int faces, int i, int j, int k) {
  T v = T(0);
  for (int b = faces & S.src_mask; b; b &= b - 1) v += src_term(S, __ffs(b) - 1, i, j, k);
  return v;
}

__device__ __forceinline__ int face_index(int f, int i, int j, int k, int nx, int ny);

// Paper-mode adjoint: the cotangent c of the observation-face node (i, j, k)
// enters its row as -tau c / M, M = h^3 halved on every axis on which the
// node lies on the outer boundary (the mirror ghost of d_n lambda = -(u - u~)).
template <typename T>
__device__ __forceinline__ T inj_term(const Slot<T>& S, int fall, int i, int j, int k, int nx, int ny) {
  if (S.inj == nullptr || !((fall >> S.obs_face) & 1)) return T(0);
  const int nb = ((fall & 3) ? 1 : 0) + ((fall & 12) ? 1 : 0) + ((fall & 48) ? 1 : 0);
  return S.inj_scale * T(1 << nb) * S.inj[face_index(S.obs_face, i, j, k, nx, ny)];
}

// field index of node (i, j, k)
template <typename T>
__device__ __forceinline__ long long lin(const StepArgs<T>& A, int i, int j, int k) {
  return (long long)i + (long long)A.px * ((long long)j + (long long)A.ny * k);
}

// index of node (i, j, k) in the FEM-owned (history) box
template <typename T>
__device__ __forceinline__ long long hidx(const StepArgs<T>& A, int i, int j, int k) {
  return (long long)(i - A.hx0) + (long long)A.hpx * ((long long)(j - A.fl[1]) + (long long)A.fn[1] * (k - A.fl[2]));
}

template <typename T>
__device__ __forceinline__ bool fem_owned(const StepArgs<T>& A, int i, int j, int k) {
  return i >= A.fl[0] && i <= A.fh[0] && j >= A.fl[1] && j <= A.fh[1] && k >= A.fl[2] &&
         k <= A.fh[2];
}

template <typename T>
__device__ __forceinline__ long long widx(const StepArgs<T>& A, int i, int j, int k) {
  return (long long)(i - A.wx0) +
         (long long)A.wpx * ((long long)(j - A.wl[1]) + (long long)A.wn[1] * (k - A.wl[2]));
}

// sum over the six axis edges of W_e (u_nb - u_c) at a FEM-owned node
template <typename T>
__device__ __forceinline__ T fem_lap(const StepArgs<T>& A, const T* __restrict__ Wb, const T* __restrict__ u, long long id,
                                     int i, int j, int k, T c, T zm, T zp) {
  const long long w = widx(A, i, j, k);
  const T* Wx = Wb;
  const T* Wy = Wb + A.wsz;
  const T* Wz = Wb + 2 * A.wsz;
  const long long wy = A.wpx;
  const long long wz = (long long)A.wpx * A.wn[1];
  return Wx[w] * (u[id + 1] - c) + Wx[w - 1] * (u[id - 1] - c) + Wy[w] * (u[id + A.px] - c) +
         Wy[w - wy] * (u[id - A.px] - c) + Wz[w] * (zp - c) + Wz[w - wz] * (zm - c);
}

// ---- the all-FEM path (HYB_FEM_TET_ALL): rows gathered over tetrahedra ----
// Coefficient a of the voxel with origin (ox, oy, oz): its value on the
// unknown voxels, 1 elsewhere (Eq. (2.3)).
template <typename T>
__device__ __forceinline__ double voxel_coef(const StepArgs<T>& A, int ox, int oy, int oz) {
  const int x = ox - A.fl[0], y = oy - A.fl[1], z = oz - A.fl[2];
  if (x >= 0 && y >= 0 && z >= 0 && x < A.un[0] && y < A.un[1] && z < A.un[2])
    return A.acoef[x + (long long)A.un[0] * (y + (long long)A.un[1] * z)];
  return 1.0;
}

template <typename T>
__device__ __forceinline__ bool lattice_interior(const StepArgs<T>& A, int i, int j, int k) {
  return i > 0 && j > 0 && k > 0 && i < A.nx - 1 && j < A.ny - 1 && k < A.nz - 1;
}

// The finite-element row of the interior node n = (i, j, k), gathered over
// the Kuhn tetrahedra of the (up to eight) voxels that have n as a corner:
// sum over those tetrahedra K of a_K K^K_{n q} (element stiffness, Sec. 7.2)
// and the lumped mass M^L_n = sum |K| / 4.  With `u` set, returns the
// Laplacian part -(M^L)^{-1} (K u)_n of Eq. (fem) (unit spacing); else the
// coefficient of row n on node m = (mi, mj, mk) (the diagonal when m = n).
template <typename T>
__device__ __noinline__ T tet_row(const StepArgs<T>& A, const T* __restrict__ u, int i, int j, int k, int mi, int mj,
                                  int mk) {
  const T c = u ? u[lin(A, i, j, k)] : T(0);
  T acc = T(0);
  double mass = 0.0;
  for (int cn = 0; cn < 8; ++cn) {
    const int ox = i - (cn & 1), oy = j - ((cn >> 1) & 1), oz = k - (cn >> 2);
    if (ox < 0 || oy < 0 || oz < 0 || ox > A.nx - 2 || oy > A.ny - 2 || oz > A.nz - 2) continue;
    const T av = (T)voxel_coef(A, ox, oy, oz);
    for (int t = 0; t < 6; ++t) {
      const int* V = A.kuhn_v + 4 * t;
      int ln = -1;
      for (int q = 0; q < 4; ++q)
        if (V[q] == cn) ln = q;
      if (ln < 0) continue;
      mass += A.kuhn[96 + t] * 0.25;
      for (int q = 0; q < 4; ++q) {
        const int cq = V[q];
        const int qi = ox + (cq & 1), qj = oy + ((cq >> 1) & 1), qk = oz + (cq >> 2);
        const T kv = av * (T)A.kuhn[16 * t + 4 * ln + q];
        if (u) {
          if (q != ln) acc += kv * (u[lin(A, qi, qj, qk)] - c);
        } else if (qi == mi && qj == mj && qk == mk) {
          acc += kv;
        }
      }
    }
  }
  return -acc / (T)mass;
}

// Coefficient of the non-absorbing row of node n on node m (Laplacian part,
// unit spacing) on the all-FEM path: the gathered FEM row on interior
// nodes; on the outer boundary the FDM row (mirror ghost: 2 on the inward
// neighbour, 1 on the in-face neighbours, -6 on the node itself).
template <typename T>
__device__ __forceinline__ T tet_coef(const StepArgs<T>& A, int ni, int nj, int nk, int mi, int mj, int mk) {
  if (lattice_interior(A, ni, nj, nk)) return tet_row<T>(A, nullptr, ni, nj, nk, mi, mj, mk);
  const int d0 = mi - ni, d1 = mj - nj, d2 = mk - nk;
  if (d0 == 0 && d1 == 0 && d2 == 0) return A.ani ? A.kdiag : T(-6);
  if (abs(d0) + abs(d1) + abs(d2) != 1) return T(0);
  const int ax = d0 ? 0 : (d1 ? 1 : 2), s = d0 + d1 + d2;
  const int c = ax == 0 ? ni : (ax == 1 ? nj : nk);
  const int n = ax == 0 ? A.nx : (ax == 1 ? A.ny : A.nz);
  const T w = ((s > 0 && c == 0) || (s < 0 && c == n - 1)) ? T(2) : T(1);
  return A.ani ? w * A.kapt[ax] : w;
}

// Pairing of the voxel with origin (i, j, k) on the all-FEM path:
// kGradPairScale sum over its tetrahedra of u^T K^K lambda (a = 1).
template <typename T>
__device__ __forceinline__ T tet_pair(const StepArgs<T>& A, const T* __restrict__ hb, const T* __restrict__ lam,
                                      int i, int j, int k) {
  T u[8], l[8];
  for (int c = 0; c < 8; ++c) {
    const int a = c & 1, b = (c >> 1) & 1, d = c >> 2;
    u[c] = hb[hidx(A, i + a, j + b, k + d)];
    l[c] = lam[lin(A, i + a, j + b, k + d)];
  }
  T acc = T(0);
  for (int t = 0; t < 6; ++t)
    for (int p = 0; p < 4; ++p)
      for (int q = 0; q < 4; ++q)
        acc += (T)A.kuhn[16 * t + 4 * p + q] * u[A.kuhn_v[4 * t + p]] * l[A.kuhn_v[4 * t + q]];
  return T(6) * acc;
}

// Laplacian part (without 1/h^2) of a non-absorbing row at any node:
// FEM stencil on FEM-owned nodes, 7-point with mirror ghosts elsewhere (on
// the all-FEM path, the gathered FEM row on every interior node).
template <typename T>
__device__ __noinline__ T row_lap(const StepArgs<T>& A, const T* __restrict__ W, const T* __restrict__ u, int i, int j,
                                  int k) {
  if (A.tet && lattice_interior(A, i, j, k)) return tet_row<T>(A, u, i, j, k, 0, 0, 0);
  const long long id = lin(A, i, j, k);
  const long long sz = (long long)A.px * A.ny;
  const T c = u[id];
  if (fem_owned(A, i, j, k)) return fem_lap(A, W, u, id, i, j, k, c, u[id - sz], u[id + sz]);
  T lx, ly, lz;
  if (i == 0) lx = T(2) * (u[id + 1] - c);
  else if (i == A.nx - 1) lx = T(2) * (u[id - 1] - c);
  else lx = (u[id - 1] - c) + (u[id + 1] - c);
  if (j == 0) ly = T(2) * (u[id + A.px] - c);
  else if (j == A.ny - 1) ly = T(2) * (u[id - A.px] - c);
  else ly = (u[id - A.px] - c) + (u[id + A.px] - c);
  if (k == 0) lz = T(2) * (u[id + sz] - c);
  else if (k == A.nz - 1) lz = T(2) * (u[id - sz] - c);
  else lz = (u[id - sz] - c) + (u[id + sz] - c);
  if (A.ani) return (A.kapt[0] * lx + A.kapt[1] * ly) + A.kapt[2] * lz;
  return (lx + ly) + lz;
}

// Coefficient of u_b^k in the absorbing row of a node on the absorbing faces
// fb (bits): r, or with per-axis steps the mean of its faces' coefficients.
template <typename T>
__device__ __forceinline__ T abc_self(const StepArgs<T>& A, int fb) {
  if (!A.ani) return A.r;
  T rs = T(0);
  for (int b = fb; b; b &= b - 1) rs += A.ra[(__ffs(b) - 1) >> 1];
  return rs / T(__popc(fb));
}

// u^{k+1} at any node, recursing into the inward neighbours of absorbing
// rows (depth D bounds the recursion: a node lies on at most 3 faces).
template <typename T, int D>
__device__ __noinline__ T fwd_new(const StepArgs<T>& A, const Slot<T>& S, int i, int j, int k) {
  const long long id = lin(A, i, j, k);
  const int fall = face_bits(i, j, k, A.nx, A.ny, A.nz);
  if constexpr (D > 0) {
    const int fb = fall & S.mask_f;
    if (fb) {
      T acc = T(0);
#pragma unroll
      for (int f = 0; f < 6; ++f) {
        if (fb & (1 << f)) {
          const int ax = f >> 1;
          const int step = (f & 1) ? -1 : 1;  // inward
          const int i1 = i + (ax == 0 ? step : 0);
          const int j1 = j + (ax == 1 ? step : 0);
          const int k1 = k + (ax == 2 ? step : 0);
          const T rf = A.ani ? A.ra[ax] : A.r;
          acc += S.cur[lin(A, i1, j1, k1)] - rf * fwd_new<T, D - 1>(A, S, i1, j1, k1);
        }
      }
      return abc_self(A, fb) * S.cur[id] + acc / T(__popc(fb));
    }
  }
  const T c = S.cur[id];
  T v = c + ((c - S.prev[id]) + A.c2 * row_lap(A, S.W, S.cur, i, j, k));
  if (fall & S.src_mask) v += src_terms(S, fall, i, j, k);
  if (S.inj) v += inj_term(S, fall, i, j, k, A.nx, A.ny);
  return v;
}

// Coefficient of the non-absorbing row of node (i,j,k) on its neighbour
// (i,j,k) + s e_ax (Laplacian part, without 1/h^2).
template <typename T>
__device__ __forceinline__ T row_coef(const StepArgs<T>& A, const T* __restrict__ W, int i, int j, int k, int ax,
                                      int s) {
  if (fem_owned(A, i, j, k)) {
    const long long w = widx(A, i, j, k);
    const long long ws = ax == 0 ? 1 : (ax == 1 ? (long long)A.wpx : (long long)A.wpx * A.wn[1]);
    return W[ax * A.wsz + (s > 0 ? w : w - ws)];
  }
  const int c = ax == 0 ? i : (ax == 1 ? j : k);
  const int n = ax == 0 ? A.nx : (ax == 1 ? A.ny : A.nz);
  const T w = ((s > 0 && c == 0) || (s < 0 && c == n - 1)) ? T(2) : T(1);
  return A.ani ? w * A.kapt[ax] : w;
}

template <typename T>
__device__ __forceinline__ T row_diag(const StepArgs<T>& A, const T* __restrict__ W, int i, int j, int k) {
  if (fem_owned(A, i, j, k)) {
    const long long w = widx(A, i, j, k);
    const long long wy = A.wpx;
    const long long wz = (long long)A.wpx * A.wn[1];
    return -(W[w] + W[w - 1] + W[A.wsz + w] + W[A.wsz + w - wy] + W[2 * A.wsz + w] +
             W[2 * A.wsz + w - wz]);
  }
  return A.ani ? A.kdiag : T(-6);
}

__device__ __forceinline__ int face_index(int f, int i, int j, int k, int nx, int ny) {
  const int ax = f >> 1;
  if (ax == 2) return i + nx * j;
  if (ax == 1) return i + nx * k;
  return j + ny * k;
}

// Right-hand side of the transposed step at node m:
// (B_j^T lambda^{j+1})_m - (C_{j+1}^T lambda^{j+2})_m + c^j_m.
template <typename T>
__device__ __noinline__ T adj_rhs(const StepArgs<T>& A, const Slot<T>& S, int i, int j, int k) {
  const T* __restrict__ l1 = S.cur;
  const long long id = lin(A, i, j, k);
  const int fbm = face_bits(i, j, k, A.nx, A.ny, A.nz);
  T rhs;
  if (fbm & S.mask_f) rhs = abc_self(A, fbm & S.mask_f) * l1[id];
  else rhs = (T(2) + A.c2 * row_diag(A, S.W, i, j, k)) * l1[id];
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int s = t ? 1 : -1;
      const int ni = i + (ax == 0 ? s : 0);
      const int nj = j + (ax == 1 ? s : 0);
      const int nk = k + (ax == 2 ? s : 0);
      if (ni < 0 || ni >= A.nx || nj < 0 || nj >= A.ny || nk < 0 || nk >= A.nz) continue;
      const long long nid = lin(A, ni, nj, nk);
      const int fbn = face_bits(ni, nj, nk, A.nx, A.ny, A.nz) & S.mask_f;
      if (fbn) {
        // absorbing row of the neighbour couples to m only when m is its
        // inward neighbour across the face on side s of axis ax
        const int f = 2 * ax + (s > 0 ? 1 : 0);
        if (fbn & (1 << f)) rhs += l1[nid] / T(__popc(fbn));
      } else {
        rhs += A.c2 * row_coef(A, S.W, ni, nj, nk, ax, -s) * l1[nid];
      }
    }
  }
  if (!(fbm & S.mask_c)) rhs -= S.prev[id];
  if (S.obs_r && ((fbm >> S.obs_face) & 1)) rhs += S.obs_r[face_index(S.obs_face, i, j, k, A.nx, A.ny)];
  return rhs;
}

// adj_rhs on the all-FEM path: the transposed row gathers the coefficients
// of every neighbouring row (the 26 nodes around m) on m.
template <typename T>
__device__ __noinline__ T adj_rhs_tet(const StepArgs<T>& A, const Slot<T>& S, int i, int j, int k) {
  const T* __restrict__ l1 = S.cur;
  const long long id = lin(A, i, j, k);
  const int fbm = face_bits(i, j, k, A.nx, A.ny, A.nz);
  T rhs;
  if (fbm & S.mask_f) rhs = abc_self(A, fbm & S.mask_f) * l1[id];
  else rhs = (T(2) + A.c2 * tet_coef(A, i, j, k, i, j, k)) * l1[id];
  for (int d = 0; d < 27; ++d) {
    const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
    if (d == 13) continue;
    const int ni = i + dx, nj = j + dy, nk = k + dz;
    if (ni < 0 || ni >= A.nx || nj < 0 || nj >= A.ny || nk < 0 || nk >= A.nz) continue;
    const long long nid = lin(A, ni, nj, nk);
    const int fbn = face_bits(ni, nj, nk, A.nx, A.ny, A.nz) & S.mask_f;
    if (fbn) {
      // an absorbing row couples to m only when m is its inward neighbour
      // across one of its absorbing faces
      if (abs(dx) + abs(dy) + abs(dz) != 1) continue;
      const int ax = dx ? 0 : (dy ? 1 : 2), s = -(dx + dy + dz);  // m = n + s e_ax
      const int f = 2 * ax + (s > 0 ? 0 : 1);
      if (fbn & (1 << f)) rhs += l1[nid] / T(__popc(fbn));
    } else {
      rhs += A.c2 * tet_coef(A, ni, nj, nk, i, j, k) * l1[nid];
    }
  }
  if (!(fbm & S.mask_c)) rhs -= S.prev[id];
  if (S.obs_r && ((fbm >> S.obs_face) & 1)) rhs += S.obs_r[face_index(S.obs_face, i, j, k, A.nx, A.ny)];
  return rhs;
}

// Inlined copy of adj_rhs (below).
// Right-hand side of the transposed step at node m:
// (B_j^T lambda^{j+1})_m - (C_{j+1}^T lambda^{j+2})_m + c^j_m.
// Inlined form of adj_rhs for the edge tiles.  Every load is issued first,
// predicated, and the row summed afterwards: the nodes of an edge tile's warp
// take different branches (faces, absorbing rows, FEM weights), and loads
// inside those branches would each wait for memory in turn.
template <typename T>
__device__ __forceinline__ T adj_rhs_inl(const StepArgs<T>& A, const Slot<T>& S, int i, int j, int k) {
  const T* __restrict__ l1 = S.cur;
  const long long id = lin(A, i, j, k);
  const int fbm = face_bits(i, j, k, A.nx, A.ny, A.nz);
  const long long wy = A.wpx, wz = (long long)A.wpx * A.wn[1];
  const bool fo = fem_owned(A, i, j, k);
  const long long w = fo ? widx(A, i, j, k) : 0;
  const T* W = S.W;
  T wd[6];  // this node's edge weights (FEM-owned nodes)
  wd[0] = fo ? W[w] : T(0);
  wd[1] = fo ? W[w - 1] : T(0);
  wd[2] = fo ? W[A.wsz + w] : T(0);
  wd[3] = fo ? W[A.wsz + w - wy] : T(0);
  wd[4] = fo ? W[2 * A.wsz + w] : T(0);
  wd[5] = fo ? W[2 * A.wsz + w - wz] : T(0);
  const T lc = l1[id];
  const T pv = S.prev[id];
  const bool obs = S.obs_r != nullptr && ((fbm >> S.obs_face) & 1);
  const T ov = obs ? S.obs_r[face_index(S.obs_face, i, j, k, A.nx, A.ny)] : T(0);
  T nb[6], cw[6];
  int nfb[6];
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int q = 2 * ax + t;
      const int s = t ? 1 : -1;
      const int ni = i + (ax == 0 ? s : 0);
      const int nj = j + (ax == 1 ? s : 0);
      const int nk = k + (ax == 2 ? s : 0);
      const bool inb = ni >= 0 && ni < A.nx && nj >= 0 && nj < A.ny && nk >= 0 && nk < A.nz;
      nb[q] = l1[inb ? lin(A, ni, nj, nk) : id];
      nfb[q] = inb ? (face_bits(ni, nj, nk, A.nx, A.ny, A.nz) & S.mask_f) : -1;
      // coefficient of the neighbour's non-absorbing row on this node (row_coef)
      const bool nfo = inb && fem_owned(A, ni, nj, nk);
      const long long ws = ax == 0 ? 1 : (ax == 1 ? wy : wz);
      const long long nw = nfo ? ax * A.wsz + (s < 0 ? widx(A, ni, nj, nk) : widx(A, ni, nj, nk) - ws) : 0;
      const T wv = nfo ? W[nw] : T(0);
      const int c = ax == 0 ? ni : (ax == 1 ? nj : nk);
      const int n = ax == 0 ? A.nx : (ax == 1 ? A.ny : A.nz);
      cw[q] = nfo ? wv : (((s < 0 && c == 0) || (s > 0 && c == n - 1)) ? T(2) : T(1));
    }
  }
  T rhs;
  if (fbm & S.mask_f) rhs = A.r * lc;
  else rhs = (T(2) + A.c2 * (fo ? -(wd[0] + wd[1] + wd[2] + wd[3] + wd[4] + wd[5]) : T(-6))) * lc;
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    if (nfb[q] < 0) continue;
    if (nfb[q]) {
      // absorbing row of the neighbour couples to m only when m is its
      // inward neighbour across the face on side s of axis ax
      const int f = 2 * (q >> 1) + (q & 1);
      if (nfb[q] & (1 << f)) rhs += nb[q] / T(__popc(nfb[q]));
    } else {
      rhs += A.c2 * cw[q] * nb[q];
    }
  }
  if (!(fbm & S.mask_c)) rhs -= pv;
  return rhs + ov;
}

// lambda^j at node m: solve E_{j-1}^T lambda^j = rhs, where E couples an
// absorbing node b to its inward neighbours with r / L_b.
template <typename T, int D>
__device__ __noinline__ T adj_new(const StepArgs<T>& A, const Slot<T>& S, int i, int j, int k) {
  T v = A.tet ? adj_rhs_tet(A, S, i, j, k) : adj_rhs(A, S, i, j, k);
  if constexpr (D > 0) {
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const int s = t ? 1 : -1;
        const int bi = i + (ax == 0 ? s : 0);
        const int bj = j + (ax == 1 ? s : 0);
        const int bk = k + (ax == 2 ? s : 0);
        if (bi < 0 || bi >= A.nx || bj < 0 || bj >= A.ny || bk < 0 || bk >= A.nz) continue;
        const int f = 2 * ax + (s > 0 ? 1 : 0);
        const int fbb = face_bits(bi, bj, bk, A.nx, A.ny, A.nz) & S.mask_e;
        if (fbb & (1 << f)) v -= ((A.ani ? A.ra[ax] : A.r) / T(__popc(fbb))) * adj_new<T, D - 1>(A, S, bi, bj, bk);
      }
    }
  }
  return v;
}

// Six times the sum over the 12 axis edges of a voxel of
// w_e (u_p - u_q)(l_p - l_q), corner c = a + 2b + 4d at offset (a, b, d);
// w_e = 1/3 on the edges at the voxel's diagonal corners 0 and 7, 1/6 on the
// others.  (The factor 6 keeps divisions out of the kernels; the host scale
// of the gradient divides it out.)
template <typename T>
__device__ __forceinline__ T pair_sum(const T u[8], const T l[8]) {
  const T d3 = (u[1] - u[0]) * (l[1] - l[0]) + (u[7] - u[6]) * (l[7] - l[6]) +
               (u[2] - u[0]) * (l[2] - l[0]) + (u[7] - u[5]) * (l[7] - l[5]) +
               (u[4] - u[0]) * (l[4] - l[0]) + (u[7] - u[3]) * (l[7] - l[3]);
  const T d6 = (u[3] - u[2]) * (l[3] - l[2]) + (u[5] - u[4]) * (l[5] - l[4]) +
               (u[3] - u[1]) * (l[3] - l[1]) + (u[6] - u[4]) * (l[6] - l[4]) +
               (u[5] - u[1]) * (l[5] - l[1]) + (u[6] - u[2]) * (l[6] - l[2]);
  return T(2) * d3 + d6;
}

// Telegraph reading: 12 times the pairing sum_i m_i lambda_i v_i of a voxel,
// v = u^{k+1} - u^{k-1} at its corners (the stored history) and m_i its lumped
// mass share of corner i in units of h^3: 1/4 on the diagonal corners 0 and
// 7, 1/12 on the others.
template <typename T>
__device__ __forceinline__ T damp_sum(const T u[8], const T l[8]) {
  const T d = u[0] * l[0] + u[7] * l[7];
  const T o = ((u[1] * l[1] + u[2] * l[2]) + (u[3] * l[3] + u[4] * l[4])) + (u[5] * l[5] + u[6] * l[6]);
  return T(3) * d + o;
}

// pair_sum with per-axis steps: the sums over the x, y and z edges weighed by
// kap (the voxel is a brick; dx_1^2 / dx_ax^2 relative to the x edges).
template <typename T>
__device__ __forceinline__ T pair_sum_ani(const StepArgs<T>& A, const T u[8], const T l[8]) {
  const T x = T(2) * ((u[1] - u[0]) * (l[1] - l[0]) + (u[7] - u[6]) * (l[7] - l[6])) +
              ((u[3] - u[2]) * (l[3] - l[2]) + (u[5] - u[4]) * (l[5] - l[4]));
  const T y = T(2) * ((u[2] - u[0]) * (l[2] - l[0]) + (u[7] - u[5]) * (l[7] - l[5])) +
              ((u[3] - u[1]) * (l[3] - l[1]) + (u[6] - u[4]) * (l[6] - l[4]));
  const T z = T(2) * ((u[4] - u[0]) * (l[4] - l[0]) + (u[7] - u[3]) * (l[7] - l[3])) +
              ((u[5] - u[1]) * (l[5] - l[1]) + (u[6] - u[2]) * (l[6] - l[2]));
  return (A.kapt[0] * x + A.kapt[1] * y) + A.kapt[2] * z;
}

// pair_sum of voxel (i,j,k): u from the FEM-owned box hb, lambda from the lattice
template <typename T>
__device__ __forceinline__ T voxel_pair(const StepArgs<T>& A, const T* __restrict__ hb,
                                        const T* __restrict__ lam, int i, int j, int k) {
  const long long hy = A.hpx;
  const long long hz = (long long)A.hpx * A.fn[1];
  const long long h0 = hidx(A, i, j, k);
  const long long ly = A.px;
  const long long lz = (long long)A.px * A.ny;
  const long long l0 = lin(A, i, j, k);
  T u[8], l[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int a = c & 1, b = (c >> 1) & 1, d = c >> 2;
    u[c] = hb[h0 + a + b * hy + d * hz];
    l[c] = lam[l0 + a + b * ly + d * lz];
  }
  return A.sdamp ? damp_sum(u, l) : pair_sum(u, l);
}

// voxel_pair with per-axis steps (the per-axis and all-node kernels)
template <typename T>
__device__ __forceinline__ T voxel_pair_ani(const StepArgs<T>& A, const T* __restrict__ hb,
                                            const T* __restrict__ lam, int i, int j, int k) {
  T u[8], l[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int a = c & 1, b = (c >> 1) & 1, d = c >> 2;
    u[c] = hb[hidx(A, i + a, j + b, k + d)];
    l[c] = lam[lin(A, i + a, j + b, k + d)];
  }
  return pair_sum_ani(A, u, l);
}

// Laplacian part (without 1/h^2) of a 7-point row with unit weights.
template <typename T>
__device__ __forceinline__ T lap7(T xm, T xp, T ym, T yp, T zm, T zp, T c) {
  return (xm - c) + (xp - c) + (ym - c) + (yp - c) + (zm - c) + (zp - c);
}

// Laplacian part of a non-absorbing row (inlined form of row_lap).
template <typename T>
__device__ __forceinline__ T row_lap_inl(const StepArgs<T>& A, const T* __restrict__ W, const T* __restrict__ u, int i,
                                         int j, int k) {
  const long long id = lin(A, i, j, k);
  const long long sz = (long long)A.px * A.ny;
  const T c = u[id];
  if (fem_owned(A, i, j, k)) return fem_lap(A, W, u, id, i, j, k, c, u[id - sz], u[id + sz]);
  const T xm = i > 0 ? u[id - 1] : u[id + 1];
  const T xp = i < A.nx - 1 ? u[id + 1] : u[id - 1];
  const T ym = j > 0 ? u[id - A.px] : u[id + A.px];
  const T yp = j < A.ny - 1 ? u[id + A.px] : u[id - A.px];
  const T zm = k > 0 ? u[id - sz] : u[id + sz];
  const T zp = k < A.nz - 1 ? u[id + sz] : u[id - sz];
  return lap7(xm, xp, ym, yp, zm, zp, c);
}

// (TET: the all-node and per-axis kernels; the all-node ones also serve the all-FEM path)
template <typename T, bool TET>
__device__ __forceinline__ void pair_if_voxel(const StepArgs<T>& A, const Slot<T>& S, int si, int i, int j,
                                              int k) {
  if (S.hist_r == nullptr) return;
  if (i < A.fl[0] || i >= A.fl[0] + A.un[0] || j < A.fl[1] || j >= A.fl[1] + A.un[1] || k < A.fl[2] ||
      k >= A.fl[2] + A.un[2])
    return;
  const long long nv = (long long)A.un[0] * A.un[1] * A.un[2];
  const long long vid = (long long)(i - A.fl[0]) +
                        (long long)A.un[0] * ((j - A.fl[1]) + (long long)A.un[1] * (k - A.fl[2]));
  if (A.refvox && A.refvox[vid]) return;
  if (TET && A.tet) A.G[(long long)si * nv + vid] += (double)tet_pair(A, S.hist_r, S.cur, i, j, k);
  else if (TET && A.ani) A.G[(long long)si * nv + vid] += (double)voxel_pair_ani(A, S.hist_r, S.cur, i, j, k);
  else A.G[(long long)si * nv + vid] += (double)voxel_pair(A, S.hist_r, S.cur, i, j, k);
}

template <typename T>
__device__ __forceinline__ long long axis_stride(const StepArgs<T>& A, int ax) {
  return ax == 0 ? 1LL : (ax == 1 ? (long long)A.px : (long long)A.px * A.ny);
}

// The "edge set" (lattices with >= 5 nodes per axis): every node whose
// coordinate is near a face (0, 1, n-2 or n-1) on at least two axes.  It is
// cut into tiles of 128 threads: tile 0 is the 4 x 4 x 4 corner block
// (threads 0..63), the other tiles are 8 consecutive positions of one of
// the 12 edge bars (4 x 4 near coordinates x 8).  Within a tile every
// absorbing coupling stays inside the tile.  Returns false for idle threads;
// q[] holds the near index (0..3 -> 0, 1, n-2, n-1) per axis (-1: mid) and
// nf the number of axes on which the node is on a face.
template <typename T>
__device__ __forceinline__ bool edge_tile_node(const StepArgs<T>& A, int blk, int t, int& i, int& j, int& k,
                                               int q[3], int& nf) {
  const int nx = A.nx, ny = A.ny, nz = A.nz;
  auto nr = [](int qq, int n) { return qq < 2 ? qq : n - 4 + qq; };
  int pos = 0, bar = -1;
  if (blk == 0) {
    if (t >= 64) return false;
    q[0] = t & 3;
    q[1] = (t >> 2) & 3;
    q[2] = t >> 4;
  } else {
    blk -= 1;
    const int bz = (nz - 4 + 7) / 8, by = (ny - 4 + 7) / 8;
    const int lo = t & 3, hi = (t >> 2) & 3;
    if (blk < bz) {
      bar = 2;
      pos = blk * 8 + (t >> 4);
      if (pos >= nz - 4) return false;
      q[0] = lo;
      q[1] = hi;
      q[2] = -1;
    } else if (blk < bz + by) {
      bar = 1;
      pos = (blk - bz) * 8 + (t >> 4);
      if (pos >= ny - 4) return false;
      q[0] = lo;
      q[1] = -1;
      q[2] = hi;
    } else {
      bar = 0;
      pos = (blk - bz - by) * 8 + (t >> 4);
      if (pos >= nx - 4) return false;
      q[0] = -1;
      q[1] = lo;
      q[2] = hi;
    }
  }
  i = q[0] < 0 ? 2 + pos : nr(q[0], nx);
  j = q[1] < 0 ? 2 + pos : nr(q[1], ny);
  k = q[2] < 0 ? 2 + pos : nr(q[2], nz);
  nf = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) nf += (q[a] == 0 || q[a] == 3) ? 1 : 0;
  (void)bar;
  return true;
}

// Thread index, inside the same tile, of the node with near index qn on
// axis ax (the other coordinates unchanged).
__device__ __forceinline__ int edge_tile_peer(int t, int blk, const int q[3], int ax, int qn) {
  if (blk == 0) {
    const int sh = 2 * ax;
    return (t & ~(3 << sh)) | (qn << sh);
  }
  // bar tiles: bits 0-1 = first near axis, bits 2-3 = second near axis
  int first = -1;
#pragma unroll
  for (int a = 0; a < 3; ++a)
    if (q[a] >= 0) {
      first = a;
      break;
    }
  const int sh = (ax == first) ? 0 : 2;
  return (t & ~(3 << sh)) | (qn << sh);
}

// Position of an interior thread.
struct Col {
  int si, i, j;
  int dxs, dys;   // -1 / +1: one node inside the low / high face of x, y; 0: not
  bool xy_fem;    // (i, j) inside the FEM-owned range
  bool xy_uv;     // (i, j) is the x-y origin of an unknown voxel
  bool xy_vox;    // ... and the step pairs
  int rz0, rz1;   // z range of the column's sparse-row nodes (rz0 > rz1: none)
};

// ---- shared-memory pipeline of the interior blocks ----
// A block stages, plane by plane and kPipe<T>::D levels ahead of its z
// march, boxes that its producer warp loads with bulk tensor copies (TMA):
// u^k on the tile and a one-node halo (Box<T>: the box starts on a 16-byte
// boundary, hx columns left of the tile, and is BX x 18), u^{k-1} on the
// same box, and on tiles that meet the FEM block the three edge-weight
// arrays and, for the transposed step, the stored u of the FEM-owned box
// (BX x 17).  Each plane lives in a ring of stages indexed by the plane
// number modulo the ring size.  The copies of a level complete on its "full"
// mbarrier; each of the eight consumer warps (the 32 x 16 tile, two rows per
// thread) waits on it, reads only shared memory and arrives on the level's
// "empty" mbarrier, on which the producer waits before it overwrites the
// level's stages.  The consumer warps thus run up to D levels apart.
// stage of plane k in a ring of N stages (k >= 0)
template <int N>
__device__ __forceinline__ int ring(int k) {
  return (int)((unsigned)k % (unsigned)N);
}

template <typename T>
struct kPipe {
  static constexpr int pow2(int n) { return n <= 1 ? 1 : 2 * pow2((n + 1) / 2); }
  static constexpr int round128(int elems) { return (int)(((elems * (int)sizeof(T) + 127) / 128) * 128 / sizeof(T)); }
  static constexpr int D = 1;             // levels in flight (tiles meeting the FEM block)
  static constexpr int SC = D + 3;        // u^k stages (planes k-1 .. k+1+D)
  static constexpr int SP = pow2(D + 1);  // u^{k-1} stages (k .. k+D)
  static constexpr int SW = D + 2;        // edge-weight stages (k-1 .. k+D)
  static constexpr int SH = D + 2;        // stored-u stages (k .. k+1+D)
  static constexpr int NB = pow2(D + 1);  // level barriers (of each kind)
  static constexpr int CS = round128(Box<T>::C);  // elements per u stage (128-byte aligned)
  static constexpr int WS = round128(Box<T>::H);  // elements per edge-weight array / stored-u stage
  static constexpr int elems = SC * CS + SP * CS + SW * 3 * WS + SH * WS;
  // Tiles off the FEM block stage only u^k and u^{k-1}: they spend the same
  // shared memory on deeper rings, DP levels ahead.
  static constexpr int deep(int d) { return (d + 4 + pow2(d + 2)) * CS <= elems ? deep(d + 1) : d; }
  static constexpr int DP = deep(D);
  static constexpr int NBX = pow2(DP + 1) > NB ? pow2(DP + 1) : NB;  // barrier pairs allocated
  static constexpr size_t bytes = sizeof(T) * (size_t)elems + 16 * NBX;
};

// Ring sizes of a tile: on the FEM block (all four rings, D levels ahead) or
// off it (DEEP: u^k and u^{k-1} only, DP levels ahead).
template <typename T, bool DEEP>
struct Ring {
  using P = kPipe<T>;
  static constexpr int D = DEEP ? P::DP : P::D;
  static constexpr int SC = D + 3;
  static constexpr int SP = P::pow2(D + 1);
  static constexpr int NB = P::pow2(D + 1);
  static_assert(DEEP ? (SC + SP) * P::CS <= P::elems : (SC == P::SC && SP == P::SP && NB == P::NB), "ring sizes");
};

// Producer side of one interior block: which boxes exist, and their issue.
template <typename T, bool DEEP>
struct Producer {
  const StepArgs<T>* A;
  const Slot<T>* S;
  T *CR, *PR, *WR, *HR;
  uint64_t* full;   // [NB]: the planes of a level have landed (one arrival: the producer, plus bytes)
  uint64_t* empty;  // [NB]: the consumer warps are done with a level (eight arrivals)
  int z0, z1, xf, yf, xw, yw, xh, yh, xp, yp;
  bool fem_tile, hist_tile, pface;  // pface: u^{k-1} with its halo (tiles holding face-adjacent nodes)
  // the planes first read at level g (the first level also reads planes
  // g - 1 and g of u^k, g - 1 of the weights and g of the stored u)
  __device__ __forceinline__ void issue(int g, bool first) const {
    using P = kPipe<T>;
    using R = Ring<T, DEEP>;
    constexpr uint32_t kCBytes = (uint32_t)(Box<T>::C * sizeof(T));
    constexpr uint32_t kPBytes = (uint32_t)(Box<T>::P * sizeof(T));
    constexpr uint32_t kWBytes = (uint32_t)(Box<T>::H * sizeof(T));
    uint64_t* bar = full + ((g - z0) & (R::NB - 1));
    const int wlo = A->wl[2], whi = A->wl[2] + A->wn[2] - 1, hlo = A->fl[2], hhi = A->fh[2];
    const bool c_on = g + 1 <= z1;
    const bool w_on = !DEEP && fem_tile && g >= wlo && g <= whi;
    const bool wm_on = !DEEP && first && fem_tile && g - 1 >= wlo && g - 1 <= whi;
    const bool h_on = !DEEP && hist_tile && g + 1 >= hlo && g + 1 <= hhi;
    const bool h0_on = !DEEP && first && hist_tile && g >= hlo && g <= hhi;
    const uint32_t bytes = kCBytes * ((c_on ? 1 : 0) + (pface ? 1 : 0) + (first ? 2 : 0)) + (pface ? 0u : kPBytes) +
                           kWBytes * (3 * ((w_on ? 1 : 0) + (wm_on ? 1 : 0)) + (h_on ? 1 : 0) + (h0_on ? 1 : 0));
    mbar_arrive_expect_tx(bar, bytes);
    if (first) {
      tma_load_3d(CR + ring<R::SC>(g - 1) * P::CS, &A->tmf, xf, yf, S->zf_cur + g - 1, bar);
      tma_load_3d(CR + ring<R::SC>(g) * P::CS, &A->tmf, xf, yf, S->zf_cur + g, bar);
    }
    if (c_on) tma_load_3d(CR + ring<R::SC>(g + 1) * P::CS, &A->tmf, xf, yf, S->zf_cur + g + 1, bar);
    if (pface)
      tma_load_3d(PR + (g & (R::SP - 1)) * P::CS, &A->tmf, xf, yf, S->zf_prev + g, bar);
    else
      tma_load_3d(PR + (g & (R::SP - 1)) * P::CS, &A->tmp, xp, yp, S->zf_prev + g, bar);
    if (wm_on) weights(g - 1, bar);
    if (w_on) weights(g, bar);
    if (h0_on) tma_load_3d(HR + ring<P::SH>(g) * P::WS, &A->tmh, xh, yh, S->zf_hist + (g - hlo), bar);
    if (h_on) tma_load_3d(HR + ring<P::SH>(g + 1) * P::WS, &A->tmh, xh, yh, S->zf_hist + (g + 1 - hlo), bar);
  }
  // stages and barriers in the block's shared memory, box origins of the
  // tile (i0 - hx, j0 - 1: multiples of 4 in x, so 16-byte aligned)
  __device__ __forceinline__ void setup(const StepArgs<T>& a, const Slot<T>& s, T* sm, uint64_t* bars, int zlo,
                                        int zhi, int i0, int j0, bool hist, bool face) {
    using P = kPipe<T>;
    using R = Ring<T, DEEP>;
    A = &a;
    S = &s;
    CR = sm;
    PR = CR + R::SC * P::CS;
    WR = DEEP ? nullptr : PR + P::SP * P::CS;
    HR = DEEP ? nullptr : WR + P::SW * 3 * P::WS;
    full = bars;
    empty = bars + P::NBX;
    z0 = zlo;
    z1 = zhi;
    xf = i0 - Box<T>::hx;
    yf = j0 - 1;
    xw = i0 - Box<T>::hx - a.wx0;
    yw = j0 - 1 - a.wl[1];
    xh = i0 - Box<T>::hx - a.hx0;
    yh = j0 - a.fl[1];
    xp = i0 - Box<T>::phx;
    yp = j0;
    pface = face;
    fem_tile = !DEEP;
    hist_tile = !DEEP && hist;
  }
  __device__ __forceinline__ void weights(int q, uint64_t* bar) const {
    using P = kPipe<T>;
    T* w = WR + ring<P::SW>(q) * 3 * P::WS;
    const int zq = q - A->wl[2];
#pragma unroll
    for (int a = 0; a < 3; ++a) tma_load_3d(w + a * P::WS, &A->tmw, xw, yw, S->zf_w + a * A->wn[2] + zq, bar);
  }
};

// One node (i, j, k) of an interior block from the staged planes: Ck, Cm, Cp
// are this node in the u^k boxes of planes k, k-1, k+1, Pk in the u^{k-1}
// box, Wk / Wm in the edge-weight arrays of planes k / k-1, Hk / Hp in the
// stored-u boxes of planes k / k+1 (at the voxel origin).  ZF: the plane is
// one step inside a z face (dzs = -1 / +1: the low / high one) and the node
// also produces the face node next to it.  Tiles without FACE hold no node
// one step inside an x or y face.
template <typename T, bool ADJ, bool FEMT, bool FACE, bool ZF, bool REF, bool TEL>
__device__ __forceinline__ void interior_node(const StepArgs<T>& A, const Slot<T>& S, T* __restrict__ gnext,
                                              const Col& C, int k, int off, int dzs, const T* Ck, const T* Cm,
                                              const T* Cp, const T* Pk, const T* Wk, const T* Wm, const T* Hk,
                                              const T* Hp, int rf, T sd) {
  using P = kPipe<T>;
  constexpr int kBoxX = Box<T>::BX;
  if (ZF && FACE && (C.dxs != 0 || C.dys != 0)) return;  // near two faces: edge tiles
  const T c2 = A.c2;
  const T c0 = Ck[0], cm = Cm[0], cp = Cp[0], pv = Pk[0];
  const T xm = Ck[-1], xp = Ck[1], ym = Ck[-kBoxX], yp = Ck[kBoxX];
  bool lf = false;
  T wxm = T(1), wxp = T(1), wym = T(1), wyp = T(1);
  if constexpr (FEMT) lf = C.xy_fem && k >= A.fl[2] && k <= A.fh[2];
  T wzm = T(1), wzp = T(1);
  T val;
  if (FEMT && lf) {
    wxm = Wk[-1];
    wxp = Wk[0];
    wym = Wk[P::WS - kBoxX];
    wyp = Wk[P::WS];
    wzp = Wk[2 * P::WS];
    wzm = Wm[2 * P::WS];
    const T lap =
        wxp * (xp - c0) + wxm * (xm - c0) + wyp * (yp - c0) + wym * (ym - c0) + wzp * (cp - c0) + wzm * (cm - c0);
    if constexpr (TEL)  // damped row (sd: the node's damping ratio)
      val = c0 + ((c0 - pv) * (T(1) - sd) + c2 * lap) / (T(1) + sd);
    else
      val = c0 + ((c0 - pv) + c2 * lap);
  } else if constexpr (sizeof(T) == 4) {  // unit weights: the neighbour sum minus 6 u^k
    val = c0 + ((c0 - pv) + c2 * ((((xm + xp) + (ym + yp)) + (cm + cp)) - T(6) * c0));
  } else {  // FP64 sums the six differences
    val = c0 + ((c0 - pv) + c2 * lap7(xm, xp, ym, yp, cm, cp, c0));
  }
  if constexpr (ZF) {  // the z face node next to this node (the rows of the x / y faces below)
    const int f = dzs > 0 ? 5 : 4;
    const T* Cb = dzs > 0 ? Cp : Cm;  // b and its in-face neighbours in the staged plane k +- 1
    const T ub = Cb[0];
    const bool abc = (S.mask_f >> f) & 1;
    const int offb = off + dzs * A.px * A.ny;
    if constexpr (!ADJ) {
      T vb;
      if (abc) {
        vb = A.r * ub + (c0 - A.r * val);
      } else {
        T lb = T(2) * (c0 - ub);
        lb += (Cb[-1] - ub) + (Cb[1] - ub);
        lb += (Cb[-kBoxX] - ub) + (Cb[kBoxX] - ub);
        vb = ub + ((ub - S.prev[offb]) + c2 * lb);  // (u^{k-1} of the face plane is not staged)
        if ((S.src_mask >> f) & 1) vb += src_term(S, f, C.i, C.j, k + dzs);
        if (S.inj && S.obs_face == f) vb += S.inj_scale * T(2) * S.inj[face_index(f, C.i, C.j, k + dzs, A.nx, A.ny)];
      }
      gnext[offb] = vb;
      if (S.obs_w && S.obs_face == f) S.obs_w[face_index(f, C.i, C.j, k + dzs, A.nx, A.ny)] = vb;
    } else {
      const T coef_mb = dzs > 0 ? wzp : wzm;
      T lb = abc ? A.r * ub : (T(2) - T(6) * c2) * ub;
      lb += c2 * coef_mb * c0;
      if (!abc) {
        lb += c2 * (Cb[-1] + Cb[1]);
        lb += c2 * (Cb[-kBoxX] + Cb[kBoxX]);
      }
      if (!((S.mask_c >> f) & 1)) lb -= S.prev[offb];
      if (S.obs_r && S.obs_face == f) lb += S.obs_r[face_index(f, C.i, C.j, k + dzs, A.nx, A.ny)];
      val += (abc ? ub : T(2) * c2 * ub) - c2 * coef_mb * ub;
      if ((S.mask_e >> f) & 1) val -= A.r * lb;
      gnext[offb] = lb;
    }
  }
  if constexpr (FACE) {
    if (C.dxs != 0 || C.dys != 0) {  // the x or y face node next to this node
      const int ax = C.dxs ? 0 : 1;
      const int sd = C.dxs ? C.dxs : C.dys;
      const int f = 2 * ax + (sd > 0 ? 1 : 0);
      const int ob = ax == 0 ? sd : sd * kBoxX;  // b relative to this node in a u box
      const int o1 = ax == 0 ? kBoxX : 1;        // the other in-plane axis in the box
      const T ub = Ck[ob];
      const bool abc = (S.mask_f >> f) & 1;
      const int offb = off + (ax == 0 ? sd : sd * A.px);
      const int bi = C.i + (ax == 0 ? sd : 0), bj = C.j + (ax == 1 ? sd : 0);
      // Forward: the absorbing row of Eq. (eq:abs2) from u^k at b and m and
      // the new value at m, or the mirror-ghost row with the source flux.
      // Transposed: b's row in closed form (no transposed absorbing coupling
      // reaches it), from lambda^{j+1} at b and m, the coefficient of m's row
      // on b and lambda^{j+2} at b.  The in-face neighbours (the other
      // in-plane axis first, then z) are read only for non-absorbing faces.
      if constexpr (!ADJ) {
        T vb;
        if (abc) {
          vb = A.r * ub + (c0 - A.r * val);
        } else {
          T lb = T(2) * (c0 - ub);
          lb += (Ck[ob - o1] - ub) + (Ck[ob + o1] - ub);
          lb += (Cm[ob] - ub) + (Cp[ob] - ub);
          vb = ub + ((ub - Pk[ob]) + c2 * lb);
          if ((S.src_mask >> f) & 1) vb += src_term(S, f, bi, bj, k);
          if (S.inj && S.obs_face == f) vb += S.inj_scale * T(2) * S.inj[face_index(f, bi, bj, k, A.nx, A.ny)];
        }
        gnext[offb] = vb;
        if (S.obs_w && S.obs_face == f) S.obs_w[face_index(f, bi, bj, k, A.nx, A.ny)] = vb;
      } else {
        const T coef_mb = ax == 0 ? (sd > 0 ? wxp : wxm) : (sd > 0 ? wyp : wym);
        T lb = abc ? A.r * ub : (T(2) - T(6) * c2) * ub;
        lb += c2 * coef_mb * c0;
        if (!abc) {
          lb += c2 * (Ck[ob - o1] + Ck[ob + o1]);
          lb += c2 * (Cm[ob] + Cp[ob]);
        }
        if (!((S.mask_c >> f) & 1)) lb -= Pk[ob];
        if (S.obs_r && S.obs_face == f) lb += S.obs_r[face_index(f, bi, bj, k, A.nx, A.ny)];
        val += (abc ? ub : T(2) * c2 * ub) - c2 * coef_mb * ub;
        if ((S.mask_e >> f) & 1) val -= A.r * lb;
        gnext[offb] = lb;
      }
    }
  }
  if (!(FEMT && lf)) {
    gnext[off] = val;
    return;
  }
  const int bo = (C.i - A.hx0) + A.hpx * ((C.j - A.fl[1]) + A.fn[1] * (k - A.fl[2]));
  // rf: the node's refinement flags (0 off the columns' refined z ranges)
  if (!(REF && (rf & 1))) {  // (the refined rows write those)
    gnext[off] = val;
    if (!ADJ && S.hist_w) S.hist_w[bo] = TEL ? val - pv : val;  // (telegraph: u^{k+1} - u^{k-1})
  }
  if constexpr (ADJ) {
    const int vz = A.un[0] * A.un[1];
    const int vid = (C.i - A.fl[0]) + A.un[0] * (C.j - A.fl[1]) + vz * (k - A.fl[2]);
    if (C.xy_vox && k < A.fl[2] + A.un[2] && !(REF && (rf & 2))) {
      const T u[8] = {Hk[0], Hk[1], Hk[kBoxX], Hk[kBoxX + 1], Hp[0], Hp[1], Hp[kBoxX], Hp[kBoxX + 1]};
      const T l[8] = {c0, xp, yp, Ck[kBoxX + 1], cp, Cp[1], Cp[kBoxX], Cp[kBoxX + 1]};
      atomicAdd(A.G + (long long)C.si * ((long long)vz * A.un[2]) + vid, (double)(TEL ? damp_sum(u, l) : pair_sum(u, l)));
    }
  }
}

// The x face column of a tile whose lanes would otherwise diverge: lanes 1
// .. 16 of the producer warp, one tile row each, compute the node m one step
// inside the face (off the FEM block: unit weights) and the face node b next
// to it, so that the consumer warps skip m.  Planes and rows next to another
// face belong to the edge tiles.  The rows are those of interior_node.
struct XFace {
  bool on;   // the tile uses the face lanes
  int mi;    // x of the nodes m (1 or nx - 2)
  int sd;    // -1 / +1: the low / high x face
  int i0, j0;
};
constexpr unsigned kFaceLanes = 0x1fffeu;  // lanes 1 .. 16 of the producer warp

template <typename T, bool ADJ, bool DEEP>
__device__ __forceinline__ void xface_levels(const StepArgs<T>& A, const Slot<T>& S, const Producer<T, DEEP>& pr,
                                             const XFace& X, int z0, int z1, long long budget) {
  using P = kPipe<T>;
  using R = Ring<T, DEEP>;
  const int r = (int)threadIdx.x - (kTileX * kTileY / 2 + 1);  // tile row 0 .. 15
  const int j = X.j0 + r;
  const bool row_on = j >= 2 && j <= A.ny - 3;
  const int f = X.sd > 0 ? 1 : 0;
  const int sd = X.sd;
  constexpr int kBoxX = Box<T>::BX;
  const int o = (r + 1) * kBoxX + (X.mi - X.i0 + Box<T>::hx);  // m in a u box
  const T c2 = A.c2;
  const bool abc = (S.mask_f >> f) & 1;
  T* __restrict__ gnext = S.next;
  const int pl = A.px * A.ny;
  int off = X.mi + A.px * j + pl * z0;
  for (int k = z0; k < z1; ++k, off += pl) {
    const int q = k - z0;
    const bool ok = mbar_wait(pr.full + (q & (R::NB - 1)), (uint32_t)((q / R::NB) & 1), budget, A.err);
    if (!__all_sync(kFaceLanes, ok)) {
      if (r == 0) atomicExch(A.err, 1);
      return;
    }
    if (row_on && k >= 2 && k <= A.nz - 3) {
      const T* Ck = pr.CR + ring<R::SC>(k) * P::CS + o;
      const T* Cm = pr.CR + ring<R::SC>(k - 1) * P::CS + o;
      const T* Cp = pr.CR + ring<R::SC>(k + 1) * P::CS + o;
      const T* Pk = pr.PR + (k & (R::SP - 1)) * P::CS + o;
      const T c0 = Ck[0], xm = Ck[-1], xp = Ck[1], ym = Ck[-kBoxX], yp = Ck[kBoxX];
      const T cm = Cm[0], cp = Cp[0], pv = Pk[0];
      T val;
      if constexpr (sizeof(T) == 4)
        val = c0 + ((c0 - pv) + c2 * ((((xm + xp) + (ym + yp)) + (cm + cp)) - T(6) * c0));
      else
        val = c0 + ((c0 - pv) + c2 * lap7(xm, xp, ym, yp, cm, cp, c0));
      const T ub = Ck[sd];
      const int offb = off + sd;
      if constexpr (!ADJ) {
        T vb;
        if (abc) {
          vb = A.r * ub + (c0 - A.r * val);
        } else {
          T lb = T(2) * (c0 - ub);
          lb += (Ck[sd - kBoxX] - ub) + (Ck[sd + kBoxX] - ub);
          lb += (Cm[sd] - ub) + (Cp[sd] - ub);
          vb = ub + ((ub - Pk[sd]) + c2 * lb);
          if ((S.src_mask >> f) & 1) vb += src_term(S, f, X.mi + sd, j, k);
          if (S.inj && S.obs_face == f) vb += S.inj_scale * T(2) * S.inj[face_index(f, X.mi + sd, j, k, A.nx, A.ny)];
        }
        gnext[offb] = vb;
        if (S.obs_w && S.obs_face == f) S.obs_w[face_index(f, X.mi + sd, j, k, A.nx, A.ny)] = vb;
      } else {
        T lb = abc ? A.r * ub : (T(2) - T(6) * c2) * ub;
        lb += c2 * c0;
        if (!abc) {
          lb += c2 * (Ck[sd - kBoxX] + Ck[sd + kBoxX]);
          lb += c2 * (Cm[sd] + Cp[sd]);
        }
        if (!((S.mask_c >> f) & 1)) lb -= Pk[sd];
        if (S.obs_r && S.obs_face == f) lb += S.obs_r[face_index(f, X.mi + sd, j, k, A.nx, A.ny)];
        val += (abc ? ub : T(2) * c2 * ub) - c2 * ub;
        if ((S.mask_e >> f) & 1) val -= A.r * lb;
        gnext[offb] = lb;
      }
      gnext[off] = val;
    }
    __syncwarp(kFaceLanes);  // the lanes' reads of level k's stages are done
    if (r == 0) mbar_arrive(pr.empty + (q & (R::NB - 1)));
  }
}

// Consumer loop of an interior block, specialised by whether the tile meets
// the FEM block (FEMT) and whether it holds nodes one step inside an x or y
// face (FACE).  Each consumer thread owns two tile rows (ty and ty + 8).
template <typename T, bool ADJ, bool FEMT, bool FACE, bool REF, bool TEL = false>
__device__ __forceinline__ void interior_levels(const StepArgs<T>& A, const Slot<T>& S, const Col (&C)[2],
                                                const Producer<T, !FEMT>& pr, const bool (&active)[2],
                                                const XFace& X, int z0, int z1) {
  using P = kPipe<T>;
  using R = Ring<T, !FEMT>;
  constexpr int D = R::D;
  constexpr int kProd = kTileX * kTileY / 2;  // the producer thread
  const int t = (int)threadIdx.x;
  const long long budget = A.wait;            // cycles a pipeline wait may take
  if (t >= kProd) {
    // Producer: the planes first read at level g overwrite stages last read
    // at level g - D - 1 (the edge-weight and stored-u rings are the
    // shortest), so they are issued once every consumer warp is done with it.
    if (t != kProd) {
      if (FACE && X.on && t <= kProd + 16) xface_levels<T, ADJ, !FEMT>(A, S, pr, X, z0, z1, budget);
      return;
    }
    for (int g = 0; g < D && z0 + g < z1; ++g) pr.issue(z0 + g, g == 0);
    int g = z0 + D;
    for (; g < z1; ++g) {
      const int q = g - D - 1 - z0;
      if (q >= 0 && !mbar_wait(pr.empty + (q & (R::NB - 1)), (uint32_t)((q / R::NB) & 1), budget, A.err)) {
        atomicExch(A.err, 1);
        break;
      }
      fence_proxy_async();
      pr.issue(g, false);
    }
    // let no copy be in flight when the block exits (the consumers may have
    // given up): wait for the last issued levels, ignoring the abort flag and
    // the pipeline's own limit (the copies complete within microseconds)
    const int no_abort = 0;
    const int issued = min(g, z1) - z0;
    for (int q = max(0, issued - R::NB); q < issued; ++q)
      mbar_wait(pr.full + (q & (R::NB - 1)), (uint32_t)((q / R::NB) & 1), kDrainCycles, &no_abort);
    return;
  }
  // Consumers: each warp waits for level k's planes, computes its nodes and
  // releases the level; warps run up to D levels apart.
  const int tx = t & 31, ty = t >> 5;
  const int nz = A.nz;
  const int pl = A.px * A.ny;
  constexpr int kBoxX = Box<T>::BX;
  const int o0 = (ty + 1) * kBoxX + (tx + Box<T>::hx);  // row 0 in a u box / edge-weight array
  const int o1 = o0 + (kTileY / 2) * kBoxX;             // row 1
  const int h0 = ty * kBoxX + (tx + Box<T>::hx);        // row 0 in a stored-u box
  const int h1 = h0 + (kTileY / 2) * kBoxX;
  // u^{k-1}: the u box layout on face tiles, else the halo-free box
  const int p0 = FACE ? o0 : ty * Box<T>::PX + (tx + Box<T>::phx);
  const int p1 = FACE ? o1 : p0 + (kTileY / 2) * Box<T>::PX;
  const bool act0 = !FACE || active[0], act1 = !FACE || active[1];  // every row of a tile off the faces is active
  T* __restrict__ gnext = S.next;
  int off0 = C[0].i + A.px * C[0].j + pl * z0;       // field offsets of the two nodes
  int off1 = off0 + (kTileY / 2) * A.px;
  // refinement flags of the two nodes, loaded one level ahead (their
  // latency then overlaps the wait for the level's planes)
  auto rflag = [&](const Col& c, int kk) -> int {
    if (!REF || kk < c.rz0 || kk > c.rz1) return 0;
    return A.rmask[(c.i - A.hx0) + A.hpx * ((c.j - A.fl[1]) + A.fn[1] * (kk - A.fl[2]))];
  };
  int rfn0 = 0, rfn1 = 0;
  if constexpr (REF) {
    rfn0 = rflag(C[0], z0);
    rfn1 = rflag(C[1], z0);
  }
  // telegraph reading: the nodes' damping ratios, likewise a level ahead
  auto sdamp = [&](const Col& c, int kk) -> T {
    if (!TEL || !c.xy_fem || kk < A.fl[2] || kk > A.fh[2]) return T(0);
    return A.sdamp[(c.i - A.hx0) + A.hpx * ((c.j - A.fl[1]) + A.fn[1] * (kk - A.fl[2]))];
  };
  T sdn0 = T(0), sdn1 = T(0);
  if constexpr (TEL) {
    sdn0 = sdamp(C[0], z0);
    sdn1 = sdamp(C[1], z0);
  }
  // ring stages of planes k - 1, k, k + 1 (rotated from level to level
  // instead of reduced modulo the ring size at every level)
  int scm = ring<R::SC>(z0 - 1), sck = ring<R::SC>(z0), scp = ring<R::SC>(z0 + 1);
  int swm = 0, swk = 0, shk = 0, shp = 0;
  if constexpr (FEMT) {
    swm = ring<P::SW>(z0 - 1);
    swk = ring<P::SW>(z0);
    shk = ring<P::SH>(z0);
    shp = ring<P::SH>(z0 + 1);
  }
  for (int k = z0; k < z1; ++k, off0 += pl, off1 += pl) {
    const int q = k - z0;
    const int rf0 = rfn0, rf1 = rfn1;
    if constexpr (REF) {
      if (k + 1 < z1) {
        rfn0 = rflag(C[0], k + 1);
        rfn1 = rflag(C[1], k + 1);
      }
    }
    const T sd0 = sdn0, sd1 = sdn1;
    if constexpr (TEL) {
      if (k + 1 < z1) {
        sdn0 = sdamp(C[0], k + 1);
        sdn1 = sdamp(C[1], k + 1);
      }
    }
    const bool ok = mbar_wait(pr.full + (q & (R::NB - 1)), (uint32_t)((q / R::NB) & 1), budget, A.err);
    if (!__all_sync(0xffffffffu, ok)) {
      if (tx == 0) atomicExch(A.err, 1);
      return;
    }
    const T* Ck = pr.CR + sck * P::CS;
    const T* Cm = pr.CR + scm * P::CS;
    const T* Cp = pr.CR + scp * P::CS;
    const T* Pk = pr.PR + (k & (R::SP - 1)) * P::CS;
    const T* Wk = nullptr;
    const T* Wm = nullptr;
    const T* Hk = nullptr;
    const T* Hp = nullptr;
    if constexpr (FEMT) {
      Wk = pr.WR + swk * 3 * P::WS;
      Wm = pr.WR + swm * 3 * P::WS;
      Hk = pr.HR + shk * P::WS;
      Hp = pr.HR + shp * P::WS;
    }
    // planes one step inside a z face also produce the face plane (block-uniform)
    const int dzs = k == 1 ? -1 : (k == nz - 2 ? 1 : 0);
    if (dzs != 0) {
      if (act0)
        interior_node<T, ADJ, FEMT, FACE, true, REF, TEL>(A, S, gnext, C[0], k, off0, dzs, Ck + o0, Cm + o0, Cp + o0,
                                                Pk + p0, Wk + o0, Wm + o0, Hk + h0, Hp + h0, rf0, sd0);
      if (act1)
        interior_node<T, ADJ, FEMT, FACE, true, REF, TEL>(A, S, gnext, C[1], k, off1, dzs, Ck + o1, Cm + o1, Cp + o1,
                                                Pk + p1, Wk + o1, Wm + o1, Hk + h1, Hp + h1, rf1, sd1);
    } else {
      if (act0)
        interior_node<T, ADJ, FEMT, FACE, false, REF, TEL>(A, S, gnext, C[0], k, off0, 0, Ck + o0, Cm + o0, Cp + o0,
                                                 Pk + p0, Wk + o0, Wm + o0, Hk + h0, Hp + h0, rf0, sd0);
      if (act1)
        interior_node<T, ADJ, FEMT, FACE, false, REF, TEL>(A, S, gnext, C[1], k, off1, 0, Ck + o1, Cm + o1, Cp + o1,
                                                 Pk + p1, Wk + o1, Wm + o1, Hk + h1, Hp + h1, rf1, sd1);
    }
    __syncwarp();  // the warp's reads of level k's stages are done
    if (tx == 0) mbar_arrive(pr.empty + (q & (R::NB - 1)));
    scm = sck;
    sck = scp;
    scp = scp + 1 == R::SC ? 0 : scp + 1;
    if constexpr (FEMT) {
      swm = swk;
      swk = swk + 1 == P::SW ? 0 : swk + 1;
      shk = shp;
      shp = shp + 1 == P::SH ? 0 : shp + 1;
    }
  }
}

// Interior part of one time level (lattices with >= 5 nodes per axis):
// 32 x 16 tiles of the nodes 1 .. n-2 and z ranges, one block per work item
// (slot, tile, z range; the host balances the items by cost): eight
// consumer warps (two tile rows per thread) and a producer warp.  Nodes one
// step inside a face also produce the face node next to them.
template <typename T, bool ADJ, bool TEL>
__device__ __forceinline__ void interior_block(const StepArgs<T>& A, int b, T* sm) {
  static_assert(kTileX == 32, "one warp per tile row");
  static_assert(kTileX * kTileY / 2 + 32 == kStepBlock, "eight consumer warps (two rows each) and a producer warp");
  using P = kPipe<T>;
  const int* item = A.items + 4 * b;  // (slot, tile, z0, z1)
  const int si = item[0];
  const int tyy = item[1] / A.ntx;
  const int txx = item[1] - tyy * A.ntx;
  const int z0 = item[2], z1 = item[3];
  const int nx = A.nx, ny = A.ny;
  if (z0 >= z1) return;  // whole block
  const int t = (int)threadIdx.x;
  const int tx = t & 31, ty = t >> 5;
  const int i0 = Box<T>::x0 + txx * kTileX, j0 = 1 + tyy * kTileY;
  const Slot<T>& S = A.s[si];
  const bool has_fem = A.fl[0] <= A.fh[0];
  const bool pairing = ADJ && S.hist_r != nullptr;
  Col C[2];
  bool active[2];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    C[r].si = si;
    C[r].i = i0 + tx;
    C[r].j = j0 + ty + r * (kTileY / 2);
    C[r].dxs = (C[r].i == 1) ? -1 : (C[r].i == nx - 2 ? 1 : 0);
    C[r].dys = (C[r].j == 1) ? -1 : (C[r].j == ny - 2 ? 1 : 0);
    active[r] = t < kTileX * kTileY / 2 && C[r].i >= 1 && C[r].i <= nx - 2 && C[r].j <= ny - 2 &&
                !(C[r].dxs != 0 && C[r].dys != 0);
    C[r].xy_fem = has_fem && C[r].i >= A.fl[0] && C[r].i <= A.fh[0] && C[r].j >= A.fl[1] && C[r].j <= A.fh[1];
    C[r].xy_uv = has_fem && C[r].i >= A.fl[0] && C[r].i < A.fl[0] + A.un[0] && C[r].j >= A.fl[1] &&
                 C[r].j < A.fl[1] + A.un[1];
    C[r].xy_vox = pairing && C[r].xy_uv;
    C[r].rz0 = 1;
    C[r].rz1 = 0;
    if (A.rzr && C[r].xy_fem) {
      const int c = (C[r].i - A.fl[0]) + A.fn[0] * (C[r].j - A.fl[1]);
      C[r].rz0 = A.rzr[2 * c];
      C[r].rz1 = A.rzr[2 * c + 1];
    }
  }
  // x face column handled by the face lanes: one x face in the tile, and
  // its column m off the FEM block
  XFace X;
  {
    const bool xlo = i0 <= 1, xhi = i0 + kTileX - 1 >= nx - 2;  // the tile holds node 1 / node nx - 2
    X.mi = xlo ? 1 : nx - 2;
    X.sd = xlo ? -1 : 1;
    X.i0 = i0;
    X.j0 = j0;
    X.on = xlo != xhi && !(has_fem && X.mi >= A.fl[0] && X.mi <= A.fh[0]);
    if (X.on) {
      active[0] = active[0] && C[0].dxs == 0;
      active[1] = active[1] && C[1].dxs == 0;
    }
  }
  // block-uniform tile kinds: an item whose planes hold no FEM-owned node
  // needs no edge weights or history and runs with the deep rings
  const bool fem_tile = has_fem && i0 <= A.fh[0] && i0 + kTileX - 1 >= A.fl[0] && j0 <= A.fh[1] &&
                        j0 + kTileY - 1 >= A.fl[1] && z0 <= A.fh[2] && z1 - 1 >= A.fl[2];
  const bool face_tile = i0 <= 1 || i0 + kTileX - 1 >= nx - 2 || j0 == 1 || j0 + kTileY - 1 >= ny - 2;
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + P::elems);
  const int tp = kTileX * kTileY / 2;  // the producer thread
  if (t == tp) {
    for (int q = 0; q < P::NBX; ++q) {
      mbar_init(full + q, 1);
      mbar_init(full + P::NBX + q, kTileX * kTileY / 2 / 32 + (X.on ? 1 : 0));  // consumer warps (+ face lanes)
    }
    mbar_init_fence();
  }
  pdl_wait();  // the previous level is complete: its output may be read, its input overwritten
  __syncthreads();
  // items whose columns hold refined-voxel corners in their z range take the
  // variant with the refined rows (block-uniform)
  const bool ref_tile =
      __syncthreads_or(fem_tile && t < kTileX * kTileY / 2 &&
                       ((C[0].rz0 <= C[0].rz1 && C[0].rz0 < z1 && C[0].rz1 >= z0) ||
                        (C[1].rz0 <= C[1].rz1 && C[1].rz0 < z1 && C[1].rz1 >= z0)));
  if (fem_tile) {
    Producer<T, false> pr;
    pr.setup(A, S, sm, full, z0, z1, i0, j0, pairing, face_tile);
    if constexpr (TEL) {  // telegraph reading (no refinement)
      if (face_tile)
        interior_levels<T, ADJ, true, true, false, true>(A, S, C, pr, active, X, z0, z1);
      else
        interior_levels<T, ADJ, true, false, false, true>(A, S, C, pr, active, X, z0, z1);
    } else if (ref_tile) {
      if (face_tile)
        interior_levels<T, ADJ, true, true, true>(A, S, C, pr, active, X, z0, z1);
      else
        interior_levels<T, ADJ, true, false, true>(A, S, C, pr, active, X, z0, z1);
    } else {
      if (face_tile)
        interior_levels<T, ADJ, true, true, false>(A, S, C, pr, active, X, z0, z1);
      else
        interior_levels<T, ADJ, true, false, false>(A, S, C, pr, active, X, z0, z1);
    }
  } else {
    Producer<T, true> pr;
    pr.setup(A, S, sm, full, z0, z1, i0, j0, false, face_tile);
    if (face_tile)
      interior_levels<T, ADJ, false, true, false>(A, S, C, pr, active, X, z0, z1);
    else
      interior_levels<T, ADJ, false, false, false>(A, S, C, pr, active, X, z0, z1);
  }
}

// Edge tile of the forward step.  Levels by the number of faces a node lies
// on: nodes on no face take their interior row, then face, edge and corner
// nodes; an absorbing row (Eq. (eq:abs2)) reads the new values of its
// inward neighbours, one level down in the same tile, from shared memory.
// Every thread of the block calls it (it synchronises); nv holds 128 values.
template <typename T>
__device__ __forceinline__ void fwd_edge_tile(const StepArgs<T>& A, int si, int blk, int t, T* nv) {
  const Slot<T>& S = A.s[si];
  int i = 0, j = 0, k = 0, nf = -1, q[3];
  const bool valid = blk < A.nedge && edge_tile_node(A, blk, t, i, j, k, q, nf);
  const long long id = valid ? lin(A, i, j, k) : 0;
  const int fall = valid ? face_bits(i, j, k, A.nx, A.ny, A.nz) : 0;
  const int fb = fall & S.mask_f;
  // u^k at the node and at its inward neighbour across each absorbing face,
  // loaded before the levels below (which then wait only on shared memory)
  const T cself = valid ? S.cur[id] : T(0);
  T cin[3];
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    const int fa = (fb >> (2 * ax)) & 3;
    cin[ax] = (valid && fa) ? S.cur[id + ((fa & 1) ? 1 : -1) * axis_stride(A, ax)] : T(0);
  }
  T plain = T(0);  // the non-absorbing row, from level-k data only
  if (valid && !fb) {
    plain = cself + ((cself - S.prev[id]) + A.c2 * row_lap_inl(A, S.W, S.cur, i, j, k));
    if (fall & S.src_mask) plain += src_terms(S, fall, i, j, k);
    if (S.inj) plain += inj_term(S, fall, i, j, k, A.nx, A.ny);
  }
  nv[t] = plain;
  __syncthreads();
  for (int level = 1; level <= 3; ++level) {
    T v = T(0);
    const bool mine = valid && fb && __popc(fall) == level;
    if (mine) {
      T acc = T(0);
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) {
        const int fa = (fb >> (2 * ax)) & 3;
        if (!fa) continue;
        const int t1 = edge_tile_peer(t, blk, q, ax, (fa & 1) ? 1 : 2);
        acc += cin[ax] - A.r * nv[t1];
      }
      v = A.r * cself + acc / T(__popc(fb));
    }
    __syncthreads();
    if (mine) nv[t] = v;
    __syncthreads();
  }
  if (!valid) return;
  const T val = nv[t];
  S.next[id] = val;
  if (S.obs_w && ((fall >> S.obs_face) & 1)) S.obs_w[face_index(S.obs_face, i, j, k, A.nx, A.ny)] = val;
  if (S.hist_w && fem_owned(A, i, j, k)) S.hist_w[hidx(A, i, j, k)] = val;
}

// Edge tile of the transposed step: every thread gathers its transposed row
// in parallel, then the transposed absorbing couplings (E^T) are resolved
// from the nodes on the most faces inwards, through shared memory.
template <typename T>
__device__ __forceinline__ void adj_edge_tile(const StepArgs<T>& A, int si, int blk, int t, T* lam) {
  const Slot<T>& S = A.s[si];
  int i = 0, j = 0, k = 0, nf = -1, q[3];
  const bool valid = blk < A.nedge && edge_tile_node(A, blk, t, i, j, k, q, nf);
  lam[t] = valid ? adj_rhs_inl(A, S, i, j, k) : T(0);
  __syncthreads();
  for (int level = 2; level >= 0; --level) {
    T v = T(0);
    const bool mine = valid && nf == level;
    if (mine) {
      v = lam[t];
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) {
        if (q[ax] != 1 && q[ax] != 2) continue;  // not one node inside a face on this axis
        const int s = q[ax] == 1 ? -1 : 1;
        const int bi = i + (ax == 0 ? s : 0), bj = j + (ax == 1 ? s : 0), bk = k + (ax == 2 ? s : 0);
        const int f = 2 * ax + (s > 0 ? 1 : 0);
        const int fbb = face_bits(bi, bj, bk, A.nx, A.ny, A.nz) & S.mask_e;
        if (!(fbb & (1 << f))) continue;
        v -= (A.r / T(__popc(fbb))) * lam[edge_tile_peer(t, blk, q, ax, q[ax] == 1 ? 0 : 3)];
      }
    }
    __syncthreads();
    if (mine) lam[t] = v;
    __syncthreads();
  }
  if (!valid) return;
  S.next[lin(A, i, j, k)] = lam[t];
  pair_if_voxel<T, false>(A, S, si, i, j, k);
}

template <typename T, bool ADJ>
__device__ __forceinline__ void refined_rows(const StepArgs<T>& A, long long t);

// One time level of every slot in one launch of kStepBlock threads per
// block: first the edge tiles (two 128-node tiles per block, so their short
// dependent chains start early), then the interior blocks, then the rows of
// the refined region (gathers of short latency-bound rows, which fill the
// slots the interior blocks free towards the end of the level).  All blocks
// read levels k, k-1 and write disjoint nodes of level k+1.
template <typename T, bool ADJ, bool TEL>
__global__ void __launch_bounds__(kStepBlock, sizeof(T) == 4 ? 4 : 2) step_kernel(const __grid_constant__ StepArgs<T> A) {
  extern __shared__ __align__(128) unsigned char hyb_smem[];  // kPipe<T>::bytes
  T* sh = reinterpret_cast<T*>(hyb_smem);
  pdl_trigger();  // the next level's launch may start its blocks
  int b = blockIdx.x;
  if (b < A.nhe) {  // two 128-node tiles; the last warp takes part in the barriers only
    pdl_wait();     // the previous level is complete
    const int ne2 = (A.nedge + 1) / 2;
    const int si = b / ne2;
    const int half = (int)(threadIdx.x >> 7);
    const int blk = half < 2 ? 2 * (b - si * ne2) + half : A.nedge;
    const int t = (int)(threadIdx.x & 127);
    if constexpr (ADJ)
      adj_edge_tile<T>(A, si, blk, t, sh + 128 * half);
    else
      fwd_edge_tile<T>(A, si, blk, t, sh + 128 * half);
    return;
  }
  b -= A.nhe;
  if (b >= A.nitems) {
    pdl_wait();
    refined_rows<T, ADJ>(A, (long long)(b - A.nitems) * kStepBlock + threadIdx.x);
    return;
  }
  interior_block<T, ADJ, TEL>(A, b, sh);
}

// Lattices with fewer than 5 nodes on some axis: every node by the generic
// rows (forward and transposed).
template <typename T>
__global__ void __launch_bounds__(128) fwd_all_kernel(const __grid_constant__ StepArgs<T> A) {
  const long long n = (long long)A.nx * A.ny * A.nz;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * A.nslots) return;
  const int si = (int)(t / n);
  const long long q = t - (long long)si * n;
  const int i = (int)(q % A.nx);
  const int j = (int)((q / A.nx) % A.ny);
  const int k = (int)(q / ((long long)A.nx * A.ny));
  const long long id = lin(A, i, j, k);
  const Slot<T>& S = A.s[si];
  const T val = fwd_new<T, 3>(A, S, i, j, k);
  S.next[id] = val;
  if (S.obs_w && ((face_bits(i, j, k, A.nx, A.ny, A.nz) >> S.obs_face) & 1))
    S.obs_w[face_index(S.obs_face, i, j, k, A.nx, A.ny)] = val;
  if (S.hist_w && fem_owned(A, i, j, k)) S.hist_w[hidx(A, i, j, k)] = val;
}

template <typename T>
__global__ void __launch_bounds__(128) adj_all_kernel(const __grid_constant__ StepArgs<T> A) {
  const long long n = (long long)A.nx * A.ny * A.nz;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * A.nslots) return;
  const int si = (int)(t / n);
  const long long q = t - (long long)si * n;
  const int i = (int)(q % A.nx);
  const int j = (int)((q / A.nx) % A.ny);
  const int k = (int)(q / ((long long)A.nx * A.ny));
  const Slot<T>& S = A.s[si];
  S.next[lin(A, i, j, k)] = adj_new<T, 3>(A, S, i, j, k);
  pair_if_voxel<T, true>(A, S, si, i, j, k);
}

// Per-axis steps: each level by two launches that partition the lattice.
// The bulk launch covers the nodes at least w nodes from every face (w = 1
// forward, 2 transposed): each thread marches kAniZ consecutive planes of one
// node column (blockIdx.x: 128-node segment of the row, blockIdx.y = j - w,
// blockIdx.z = slot * chunks + chunk), keeping u of the planes below and
// above in registers, and takes their plain rows, which need no face logic;
// the shell launch enumerates the other nodes (the w layers next to each
// face) and takes them through the generic rows.
constexpr int kAniZ = 8;

template <typename T, int W>
__device__ __forceinline__ bool ani_bulk_column(const StepArgs<T>& A, int& i, int& j, int& k0, int& k1, int& si) {
  i = W + (int)(blockIdx.x * blockDim.x + threadIdx.x);
  j = W + (int)blockIdx.y;
  const int chunks = (A.nz - 2 * W + kAniZ - 1) / kAniZ;
  si = (int)blockIdx.z / chunks;
  k0 = W + ((int)blockIdx.z - si * chunks) * kAniZ;
  k1 = min(k0 + kAniZ, A.nz - W);  // exclusive
  return i <= A.nx - 1 - W;
}

// Nodes of the shell of width W of one slot: the W planes at each z face,
// then the W rows at each y face of the remaining planes, then the W nodes
// at each x face of the remaining rows.
template <typename T, int W>
__device__ __forceinline__ long long ani_shell_count(const StepArgs<T>& A) {
  return 2LL * W * ((long long)A.nx * A.ny + (long long)A.nx * (A.nz - 2 * W) +
                    (long long)(A.ny - 2 * W) * (A.nz - 2 * W));
}

template <typename T, int W>
__device__ __forceinline__ bool ani_shell_node(const StepArgs<T>& A, int& i, int& j, int& k, int& si) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long cnt = ani_shell_count<T, W>(A);
  if (t >= cnt * A.nslots) return false;
  si = (int)(t / cnt);
  long long r = t - (long long)si * cnt;
  const long long pa = 2LL * W * A.nx * A.ny;
  const long long pb = 2LL * W * A.nx * (A.nz - 2 * W);
  auto layer = [](int q, int n) { return q < W ? q : n - 2 * W + q; };  // q in [0, 2W)
  if (r < pa) {
    i = (int)(r % A.nx);
    r /= A.nx;
    j = (int)(r % A.ny);
    k = layer((int)(r / A.ny), A.nz);
  } else if ((r -= pa) < pb) {
    i = (int)(r % A.nx);
    r /= A.nx;
    j = layer((int)(r % (2 * W)), A.ny);
    k = W + (int)(r / (2 * W));
  } else {
    r -= pb;
    i = layer((int)(r % (2 * W)), A.nx);
    r /= 2 * W;
    j = W + (int)(r % (A.ny - 2 * W));
    k = W + (int)(r / (A.ny - 2 * W));
  }
  return true;
}

// Forward: bulk = every node off the faces (lattice rows with kap, FEM rows
// with the edge weights, which carry kap), shell = the face nodes.
template <typename T>
__global__ void __launch_bounds__(128) ani_fwd_bulk_kernel(const __grid_constant__ StepArgs<T> A) {
  int i, j, k0, k1, si;
  if (!ani_bulk_column<T, 1>(A, i, j, k0, k1, si)) return;
  const Slot<T>& S = A.s[si];
  const long long sz = (long long)A.px * A.ny;
  const T* __restrict__ u = S.cur;
  long long id = lin(A, i, j, k0);
  T zm = u[id - sz], c = u[id];
  const bool col_fem = i >= A.fl[0] && i <= A.fh[0] && j >= A.fl[1] && j <= A.fh[1];
  for (int k = k0; k < k1; ++k, id += sz) {
    const T zp = u[id + sz];
    const bool fo = col_fem && k >= A.fl[2] && k <= A.fh[2];
    T lap;
    if (fo) {
      lap = fem_lap(A, S.W, u, id, i, j, k, c, zm, zp);
    } else {
      const T lx = (u[id - 1] - c) + (u[id + 1] - c);
      const T ly = (u[id - A.px] - c) + (u[id + A.px] - c);
      const T lz = (zm - c) + (zp - c);
      lap = (A.kapt[0] * lx + A.kapt[1] * ly) + A.kapt[2] * lz;
    }
    const T val = c + ((c - S.prev[id]) + A.c2 * lap);
    S.next[id] = val;
    if (fo && S.hist_w) S.hist_w[hidx(A, i, j, k)] = val;
    zm = c;
    c = zp;
  }
}

template <typename T>
__global__ void __launch_bounds__(128) ani_fwd_shell_kernel(const __grid_constant__ StepArgs<T> A) {
  int i, j, k, si;
  if (!ani_shell_node<T, 1>(A, i, j, k, si)) return;
  const Slot<T>& S = A.s[si];
  const long long id = lin(A, i, j, k);
  const T val = fwd_new<T, 3>(A, S, i, j, k);
  S.next[id] = val;
  if (S.obs_w && ((face_bits(i, j, k, A.nx, A.ny, A.nz) >> S.obs_face) & 1))
    S.obs_w[face_index(S.obs_face, i, j, k, A.nx, A.ny)] = val;
}

// Transposed step: bulk = every node two or more nodes from the faces (no
// absorbing row among its neighbours, no observation), its transposed row
// gathered from the neighbours' rows (edge weight of a FEM-owned neighbour,
// kap of a lattice one) in the order of adj_rhs, plus the voxel pairing;
// shell = the nodes within one node of a face.
template <typename T>
__global__ void __launch_bounds__(128, 8) ani_adj_bulk_kernel(const __grid_constant__ StepArgs<T> A) {
  int i, j, k0, k1, si;
  if (!ani_bulk_column<T, 2>(A, i, j, k0, k1, si)) return;
  const Slot<T>& S = A.s[si];
  const long long sz = (long long)A.px * A.ny;
  const T* __restrict__ l1 = S.cur;
  long long id = lin(A, i, j, k0);
  T zm = l1[id - sz], c = l1[id];
  // columns next to the FEM block: some rows around them carry edge weights
  const bool col_near = i >= A.fl[0] - 1 && i <= A.fh[0] + 1 && j >= A.fl[1] - 1 && j <= A.fh[1] + 1;
  const T cx = A.c2 * A.kapt[0], cy = A.c2 * A.kapt[1], cz = A.c2 * A.kapt[2];
  for (int k = k0; k < k1; ++k, id += sz) {
    const T zp = l1[id + sz];
    T rhs;
    if (col_near && k >= A.fl[2] - 1 && k <= A.fh[2] + 1) {
      rhs = (T(2) + A.c2 * row_diag(A, S.W, i, j, k)) * c;
      rhs += A.c2 * row_coef(A, S.W, i - 1, j, k, 0, 1) * l1[id - 1];
      rhs += A.c2 * row_coef(A, S.W, i + 1, j, k, 0, -1) * l1[id + 1];
      rhs += A.c2 * row_coef(A, S.W, i, j - 1, k, 1, 1) * l1[id - A.px];
      rhs += A.c2 * row_coef(A, S.W, i, j + 1, k, 1, -1) * l1[id + A.px];
      rhs += A.c2 * row_coef(A, S.W, i, j, k - 1, 2, 1) * zm;
      rhs += A.c2 * row_coef(A, S.W, i, j, k + 1, 2, -1) * zp;
    } else {  // the same sums with every coefficient a lattice one
      rhs = (T(2) + A.c2 * A.kdiag) * c;
      rhs += cx * l1[id - 1];
      rhs += cx * l1[id + 1];
      rhs += cy * l1[id - A.px];
      rhs += cy * l1[id + A.px];
      rhs += cz * zm;
      rhs += cz * zp;
    }
    S.next[id] = rhs - S.prev[id];
    pair_if_voxel<T, true>(A, S, si, i, j, k);
    zm = c;
    c = zp;
  }
}

template <typename T>
__global__ void __launch_bounds__(128) ani_adj_shell_kernel(const __grid_constant__ StepArgs<T> A) {
  int i, j, k, si;
  if (!ani_shell_node<T, 2>(A, i, j, k, si)) return;
  const Slot<T>& S = A.s[si];
  S.next[lin(A, i, j, k)] = adj_new<T, 3>(A, S, i, j, k);
  pair_if_voxel<T, true>(A, S, si, i, j, k);
}

template <typename T>
__global__ void pair_kernel(const __grid_constant__ StepArgs<T> A, const T* __restrict__ hist,
                            const T* __restrict__ lam, double* __restrict__ grad) {
  const long long nv = (long long)A.un[0] * A.un[1] * A.un[2];
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nv) return;
  const int x = (int)(t % A.un[0]);
  const long long r = t / A.un[0];
  const int y = (int)(r % A.un[1]);
  const int z = (int)(r / A.un[1]);
  if (A.refvox && A.refvox[t]) return;
  const int i = A.fl[0] + x, j = A.fl[1] + y, k = A.fl[2] + z;
  grad[t] += (double)(A.tet ? tet_pair(A, hist, lam, i, j, k)
                             : (A.ani ? voxel_pair_ani(A, hist, lam, i, j, k) : voxel_pair(A, hist, lam, i, j, k)));
}

// Refined region of one time level, in the trailing blocks of the step
// launch (one thread per row), the same rows for the forward and the
// mass-scaled adjoint.  A corner n of refined voxels: the Kuhn stencil row
// lapW (the edge weights over the voxels around n) corrected on every refined
// voxel v around n by a_v (K9 - K8) of n's corner in v, which couples the
// voxel's diagonal corners 0 and 7 to its six others, the six others to 0
// and 7, and every corner to the centre; divided by n's lumped mass in units
// of h^3.  A centre c of voxel v: a_v K9 of the centre on the eight corners
// over its mass.  Then u^{k+1} = u^k + ((u^k - u^{k-1}) + tau^2/h^2 lap).
// Every load of a row is issued before the row is summed.
template <typename T, bool ADJ>
__device__ __forceinline__ void refined_corner(const StepArgs<T>& A, const Slot<T>& S, int r) {
  const uint2 pos = A.rpos[r];
  const int i = (int)(pos.x & 0xffffu), j = (int)(pos.x >> 16), k = (int)pos.y;
  const long long sy = A.px, sz = (long long)A.px * A.ny;
  const long long id = i + sy * j + sz * k;
  const T* __restrict__ u = S.cur;
  // the node's 3 x 3 x 3 neighbourhood (index (dx+1) + 3 (dy+1) + 9 (dz+1)):
  // a refined voxel's K9 - K8 couples n only to the six face neighbours
  // (which the stencil reads too) and to the six neighbours across the
  // diagonals of the coordinate planes with equal signs; a corner of a
  // refined voxel lies inside the FEM block, so all of them are lattice nodes
  T nb[27];
#pragma unroll
  for (int q = 0; q < 27; ++q) nb[q] = T(0);
  nb[13] = u[id];
  nb[12] = u[id - 1];
  nb[14] = u[id + 1];
  nb[10] = u[id - sy];
  nb[16] = u[id + sy];
  nb[4] = u[id - sz];
  nb[22] = u[id + sz];
  nb[9] = u[id - 1 - sy];
  nb[17] = u[id + 1 + sy];
  nb[3] = u[id - 1 - sz];
  nb[23] = u[id + 1 + sz];
  nb[1] = u[id - sy - sz];
  nb[25] = u[id + sy + sz];
  const T c0 = nb[13], pv = S.prev[id];
  const long long w = widx(A, i, j, k);
  const T* Wx = S.W;
  const T* Wy = S.W + A.wsz;
  const T* Wz = S.W + 2 * A.wsz;
  const long long wy = A.wpx, wz = (long long)A.wpx * A.wn[1];
  const T lapW = Wx[w] * (nb[14] - c0) + Wx[w - 1] * (nb[12] - c0) + Wy[w] * (nb[16] - c0) +
                 Wy[w - wy] * (nb[10] - c0) + Wz[w] * (nb[22] - c0) + Wz[w - wz] * (nb[4] - c0);
  // the eight voxels around n (n is corner c of the voxel with origin n - c)
  const int ox = i - A.fl[0], oy = j - A.fl[1], oz = k - A.fl[2];
  const int v0 = ox + A.un[0] * (oy + A.un[1] * oz), vy = A.un[0], vz = A.un[0] * A.un[1];
  int rc[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int dx = c & 1, dy = (c >> 1) & 1, dz = c >> 2;
    const bool in = ox - dx >= 0 && oy - dy >= 0 && oz - dz >= 0 && ox - dx < A.un[0] && oy - dy < A.un[1] &&
                    oz - dz < A.un[2];
    rc[c] = in ? A.rcid[v0 - dx - dy * vy - dz * vz] : -1;
  }
  T corr = T(0), mass = T(0);
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int dx = c & 1, dy = (c >> 1) & 1, dz = c >> 2;
    const bool ref = rc[c] >= 0;
    mass += ref ? A.rm9[c] : A.rm8[c];
    const T av = ref ? S.avox[v0 - dx - dy * vy - dz * vz] : T(0);
    const T uc = ref ? S.ccur[rc[c]] : c0;
    T sv = A.rdK[9 * c + 8] * (uc - c0);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const bool diag_c = c == 0 || c == 7, diag_q = q == 0 || q == 7;
      if (q == c || diag_c == diag_q) continue;
      const int o = ((q & 1) - dx + 1) + 3 * (((q >> 1) & 1) - dy + 1) + 9 * ((q >> 2) - dz + 1);
      sv += A.rdK[9 * c + q] * (nb[o] - c0);
    }
    corr += av * sv;
  }
  const T val = c0 + ((c0 - pv) + A.c2 * ((lapW - corr) / mass));
  S.next[id] = val;
  if (!ADJ && S.hist_w) S.hist_w[hidx(A, i, j, k)] = val;
}

// Pairing sum u^T K9 lambda over a refined voxel's 8 corners and centre
// (index 8), K9 the stiffness of the refined unit voxel (a = 1).
template <typename T, typename K>
__device__ __forceinline__ T refined_pair_sum(const T (&u)[9], const T (&l)[9], const K* __restrict__ k9) {
  T acc = T(0);
#pragma unroll
  for (int p = 0; p < 9; ++p) {
    T row = T(0);
#pragma unroll
    for (int q = 0; q < 9; ++q) row += (T)k9[p * 9 + q] * l[q];
    acc += u[p] * row;
  }
  return acc;
}

// Centre row of refined voxel v (centre order); in the transposed step with
// pairing the same thread also adds the voxel's pairing of (u^j, lambda^{j+1})
// to slot si's gradient, from the lambda values the row has loaded.
template <typename T, bool ADJ>
__device__ __forceinline__ void refined_centre(const StepArgs<T>& A, const Slot<T>& S, int v, int si) {
  const int vid = A.refvox_id[v];
  const uint2 xyz = A.rvxyz[v];
  const int x = (int)(xyz.x & 0xffffu), y = (int)(xyz.x >> 16), z = (int)xyz.y;
  const long long l0 = lin(A, A.fl[0] + x, A.fl[1] + y, A.fl[2] + z);
  const long long sy = A.px, sz = (long long)A.px * A.ny;
  T q[9];
#pragma unroll
  for (int c = 0; c < 8; ++c) q[c] = S.cur[l0 + (c & 1) + ((c >> 1) & 1) * sy + (c >> 2) * sz];
  const T uc = S.ccur[v], up = S.cprev[v], av = S.avox[vid];
  q[8] = uc;
  T sv = T(0);
#pragma unroll
  for (int c = 0; c < 8; ++c) sv += A.rK9[72 + c] * (q[c] - uc);
  const T vc = uc + ((uc - up) - A.c2 * av * sv / A.rm9[8]);
  S.cnext[v] = vc;
  if (!ADJ && S.chist_w) S.chist_w[v] = vc;
  if constexpr (ADJ) {
    if (!S.hist_r) return;
    const long long h0 = hidx(A, A.fl[0] + x, A.fl[1] + y, A.fl[2] + z);
    const long long hy = A.hpx, hz = (long long)A.hpx * A.fn[1];
    T u[9];
#pragma unroll
    for (int c = 0; c < 8; ++c) u[c] = S.hist_r[h0 + (c & 1) + ((c >> 1) & 1) * hy + (c >> 2) * hz];
    u[8] = S.chist_r[v];
    const long long nv = (long long)A.un[0] * A.un[1] * A.un[2];
    // the unit-voxel K9 from the launch parameters (kGradPairScale times the pairing, as the other kernels)
    // the only update of this entry in the launch: a reduction without return needs no load
    atomicAdd(A.G + (long long)si * nv + vid, (double)(T(kGradPairScale) * refined_pair_sum(u, q, A.rK9)));
  }
}

// Threads of the refined trailing blocks, per slot: the corner rows, then
// the centre rows (with the transposed step's pairing of their voxels).
template <typename T, bool ADJ>
__device__ __forceinline__ void refined_rows(const StepArgs<T>& A, long long t) {
  const int per = A.nrl + A.nref;
  if (t >= (long long)per * A.nslots) return;
  const int si = (int)(t / per);
  const int r = (int)(t - (long long)si * per);
  const Slot<T>& S = A.s[si];
  if (r < A.nrl)
    refined_corner<T, ADJ>(A, S, r);
  else
    refined_centre<T, ADJ>(A, S, r - A.nrl, si);
}

// Pairing of refined voxel v at level 0 (the level-0 kernel): u^T K9 lambda
// over its 8 corners and centre, K9 the stiffness of the refined unit voxel
// (a = 1); the host scales the sum like the structured pairing.
template <typename T, typename K>
__device__ __forceinline__ T refined_pair(const StepArgs<T>& A, int v, const T* __restrict__ hb,
                                          const T* __restrict__ chb, const T* __restrict__ lam,
                                          const T* __restrict__ clam, const K* __restrict__ k9) {
  const int uid = A.refvox_id[v];
  const int x = uid % A.un[0], y = (uid / A.un[0]) % A.un[1], z = uid / (A.un[0] * A.un[1]);
  const int i = A.fl[0] + x, j = A.fl[1] + y, k = A.fl[2] + z;
  const long long hy = A.hpx, hz = (long long)A.hpx * A.fn[1];
  const long long h0 = hidx(A, i, j, k);
  const long long l0 = lin(A, i, j, k);
  const long long ly = A.px, lz = (long long)A.px * A.ny;
  T u[9], l[9];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int a = c & 1, b = (c >> 1) & 1, d = c >> 2;
    u[c] = hb[h0 + a + b * hy + d * hz];
    l[c] = lam[l0 + a + b * ly + d * lz];
  }
  u[8] = chb[v];
  l[8] = clam[v];
  return refined_pair_sum(u, l, k9);
}

template <typename T>
__global__ void refined_pair_kernel(const __grid_constant__ StepArgs<T> A) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)A.nref * A.nslots) return;
  const int si = (int)(t / A.nref);
  const int v = (int)(t - (long long)si * A.nref);
  const Slot<T>& S = A.s[si];
  const long long nv = (long long)A.un[0] * A.un[1] * A.un[2];
  A.G[(long long)si * nv + A.refvox_id[v]] += (double)refined_pair(A, v, S.hist_r, S.chist_r, S.cur, S.ccur, A.k9);
}

// Damping ratio of the telegraph reading per FEM-owned node (one thread per
// node of the FEM-owned box): s_i = (tau / 2) sum_v sigma_v m_{v,i} over the
// eight voxels with a corner at i (sigma = 0 off the unknown voxels).
template <typename T>
__global__ void set_damp_kernel(const __grid_constant__ StepArgs<T> A, T* __restrict__ sd,
                                const double* __restrict__ sigma, double dt, int* flag) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nv = (long long)A.un[0] * A.un[1] * A.un[2];
  if (t < nv) {
    const double v = sigma[t];
    if (!(v >= 0.0) || !(v <= 1e300)) atomicExch(flag, 1);
  }
  const long long nown = (long long)A.fn[0] * A.fn[1] * A.fn[2];
  if (t >= nown) return;
  const int x = (int)(t % A.fn[0]), y = (int)((t / A.fn[0]) % A.fn[1]), z = (int)(t / ((long long)A.fn[0] * A.fn[1]));
  double acc = 0.0;
  for (int c = 0; c < 8; ++c) {  // node (x, y, z) is corner c of the voxel with origin (x, y, z) - c
    const int ox = x - (c & 1), oy = y - ((c >> 1) & 1), oz = z - (c >> 2);
    if (ox < 0 || oy < 0 || oz < 0 || ox >= A.un[0] || oy >= A.un[1] || oz >= A.un[2]) continue;
    const double sv = sigma[ox + (long long)A.un[0] * (oy + (long long)A.un[1] * oz)];
    acc += sv * ((c == 0 || c == 7) ? 0.25 : 1.0 / 12.0);
  }
  sd[hidx(A, A.fl[0] + x, A.fl[1] + y, A.fl[2] + z)] = (T)(0.5 * dt * acc);
}

template <typename T>
__global__ void set_coef_kernel(const __grid_constant__ StepArgs<T> A, T* __restrict__ W, T* __restrict__ avox,
                                const double* __restrict__ a, double a_max, int* flag) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nv = (long long)A.un[0] * A.un[1] * A.un[2];
  if (t < nv) {
    const double v = a[t];
    if (!(v <= a_max * (1.0 + 1e-12)) || !(v == v)) atomicExch(flag, 1);
    if (avox) avox[t] = (T)v;
  }
  if (t >= A.wsz) return;
  const int p[3] = {A.wx0 + (int)(t % A.wpx), A.wl[1] + (int)((t / A.wpx) % A.wn[1]),
                    A.wl[2] + (int)(t / ((long long)A.wpx * A.wn[1]))};
  const bool in_box = p[0] >= A.wl[0] && p[0] <= A.wl[0] + A.wn[0] - 1;  // else row padding
  for (int ax = 0; ax < 3; ++ax) {
    double w = 0.0;
    if (in_box && p[ax] + 1 <= A.wl[ax] + A.wn[ax] - 1) {
      const int P = ax == 0 ? 1 : 0;
      const int Q = ax == 2 ? 1 : 2;
      for (int bp = 0; bp < 2; ++bp) {
        for (int bq = 0; bq < 2; ++bq) {
          int v[3] = {p[0], p[1], p[2]};
          v[P] -= bp;
          v[Q] -= bq;
          double av = 1.0;
          if (v[0] >= A.fl[0] && v[0] < A.fl[0] + A.un[0] && v[1] >= A.fl[1] &&
              v[1] < A.fl[1] + A.un[1] && v[2] >= A.fl[2] && v[2] < A.fl[2] + A.un[2]) {
            av = a[(long long)(v[0] - A.fl[0]) +
                   (long long)A.un[0] * ((v[1] - A.fl[1]) + (long long)A.un[1] * (v[2] - A.fl[2]))];
          }
          w += av * (bp == bq ? (1.0 / 3.0) : (1.0 / 6.0));
        }
      }
    }
    W[ax * A.wsz + t] = (T)(A.ani ? w * A.kap[ax] : w);
  }
}

template <typename T>
__global__ void extract_owned_kernel(const __grid_constant__ StepArgs<T> A, const T* __restrict__ f,
                                     T* __restrict__ box) {
  const long long n = (long long)A.fn[0] * A.fn[1] * A.fn[2];
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int x = (int)(t % A.fn[0]);
  const long long r = t / A.fn[0];
  const int y = (int)(r % A.fn[1]);
  const int z = (int)(r / A.fn[1]);
  box[hidx(A, A.fl[0] + x, A.fl[1] + y, A.fl[2] + z)] = f[lin(A, A.fl[0] + x, A.fl[1] + y, A.fl[2] + z)];
}

template <typename T>
__global__ void extract_face_kernel(const __grid_constant__ StepArgs<T> A, const T* __restrict__ f, int face,
                                    T* __restrict__ row) {
  const int ax = face >> 1;
  const int np = ax == 0 ? A.ny : A.nx, nq = ax == 2 ? A.ny : A.nz;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= np * nq) return;
  const int cp = t % np, cq = t / np;
  const int c = (face & 1) ? (ax == 0 ? A.nx : (ax == 1 ? A.ny : A.nz)) - 1 : 0;
  const int i = ax == 0 ? c : cp, j = ax == 1 ? c : (ax == 0 ? cp : cq), k = ax == 2 ? c : cq;
  row[t] = f[lin(A, i, j, k)];
}

}  // namespace

template <typename T>
void launch_extract_face(const StepArgs<T>& a, const T* field, int f, T* row, cudaStream_t st) {
  const int ax = f >> 1;
  const int n = (ax == 0 ? a.ny : a.nx) * (ax == 2 ? a.ny : a.nz);
  extract_face_kernel<T><<<(n + 255) / 256, 256, 0, st>>>(a, field, f, row);
}

template <typename T, bool ADJ>
int launch_step(const StepArgs<T>& a, cudaStream_t st) {
  if (a.small) {
    const int w = ADJ ? 2 : 1;  // shell width
    if (a.ani && !a.tet && a.nx >= 5 && a.ny >= 5 && a.nz >= 5 && a.ny <= 65535 &&
        (long long)(a.nz - 2 * w) * a.nslots <= 65535) {
      const dim3 grid((unsigned)((a.nx - 2 * w + 127) / 128), (unsigned)(a.ny - 2 * w),
                      (unsigned)(((a.nz - 2 * w + kAniZ - 1) / kAniZ) * a.nslots));
      const long long shell = 2LL * w *
                              ((long long)a.nx * a.ny + (long long)a.nx * (a.nz - 2 * w) +
                               (long long)(a.ny - 2 * w) * (a.nz - 2 * w)) * a.nslots;
      const unsigned sgrid = (unsigned)((shell + 127) / 128);
      if (ADJ) {
        ani_adj_bulk_kernel<T><<<grid, 128, 0, st>>>(a);
        ani_adj_shell_kernel<T><<<sgrid, 128, 0, st>>>(a);
      } else {
        ani_fwd_bulk_kernel<T><<<grid, 128, 0, st>>>(a);
        ani_fwd_shell_kernel<T><<<sgrid, 128, 0, st>>>(a);
      }
      return 2;
    }
    const long long n = (long long)a.nx * a.ny * a.nz * a.nslots;
    if (ADJ)
      adj_all_kernel<T><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(a);
    else
      fwd_all_kernel<T><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(a);
    return 1;
  }
  StepArgs<T> b = a;
  b.nhe = ((a.nedge + 1) / 2) * a.nslots;
  const long long nref_threads = (long long)(a.nrl + a.nref) * a.nslots;
  b.nhr = (int)((nref_threads + kStepBlock - 1) / kStepBlock);
  const long long grid = (long long)b.nhe + b.nhr + a.nitems;
  // programmatic dependent launch: this level's blocks may start while the
  // previous step launch drains (they wait for it before touching its data)
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kStepBlock);
  cfg.dynamicSmemBytes = kPipe<T>::bytes;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (a.sdamp)
    cudaLaunchKernelEx(&cfg, step_kernel<T, ADJ, true>, b);
  else
    cudaLaunchKernelEx(&cfg, step_kernel<T, ADJ, false>, b);
  return 1;
}

template <typename T>
int launch_forward_step(const StepArgs<T>& a, cudaStream_t st) {
  return launch_step<T, false>(a, st);
}

template <typename T>
int launch_adjoint_step(const StepArgs<T>& a, cudaStream_t st) {
  return launch_step<T, true>(a, st);
}

template <typename T, bool ADJ>
int step_occupancy() {
  int n = 0;
  if (cudaFuncSetAttribute(step_kernel<T, ADJ, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kPipe<T>::bytes) != cudaSuccess ||
      cudaFuncSetAttribute(step_kernel<T, ADJ, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kPipe<T>::bytes) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_kernel<T, ADJ, false>, kStepBlock, kPipe<T>::bytes) !=
          cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return n > 0 ? n : 1;
}

int step_blocks_per_sm(int precision, int adjoint) {
  if (precision == HYB_FP32) return adjoint ? step_occupancy<float, true>() : step_occupancy<float, false>();
  return adjoint ? step_occupancy<double, true>() : step_occupancy<double, false>();
}

template <typename T>
void launch_refined_pair(const StepArgs<T>& a, cudaStream_t st) {
  const long long n = (long long)a.nref * a.nslots;
  if (n == 0) return;
  refined_pair_kernel<T><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(a);
}

template <typename T>
void launch_pair(const StepArgs<T>& a, const T* hist, const T* lam, cudaStream_t st) {
  const long long nv = (long long)a.un[0] * a.un[1] * a.un[2];
  if (nv == 0) return;
  pair_kernel<T><<<(unsigned)((nv + 255) / 256), 256, 0, st>>>(a, hist, lam, a.G);
}

template <typename T>
void launch_set_damp(const StepArgs<T>& a, T* sdamp, const double* sigma, double dt, int* flag, cudaStream_t st) {
  const long long nv = (long long)a.un[0] * a.un[1] * a.un[2];
  const long long nown = (long long)a.fn[0] * a.fn[1] * a.fn[2];
  const long long n = nown > nv ? nown : nv;
  if (n == 0) return;
  set_damp_kernel<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, sdamp, sigma, dt, flag);
}

template <typename T>
void launch_set_coef(const StepArgs<T>& a, T* W, T* avox, const double* acoef, double a_max, int* flag,
                     cudaStream_t st) {
  const long long nv = (long long)a.un[0] * a.un[1] * a.un[2];
  const long long n = a.wsz > nv ? a.wsz : nv;
  if (n == 0) return;
  set_coef_kernel<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, W, avox, acoef, a_max, flag);
}

template <typename T>
void launch_extract_owned(const StepArgs<T>& a, const T* field, T* box, cudaStream_t st) {
  const long long n = (long long)a.fn[0] * a.fn[1] * a.fn[2];
  if (n == 0) return;
  extract_owned_kernel<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, field, box);
}

#define HYB_INSTANTIATE(T)                                                                       \
  template int launch_forward_step<T>(const StepArgs<T>&, cudaStream_t);                         \
  template int launch_adjoint_step<T>(const StepArgs<T>&, cudaStream_t);                         \
  template void launch_pair<T>(const StepArgs<T>&, const T*, const T*, cudaStream_t);            \
  template void launch_set_coef<T>(const StepArgs<T>&, T*, T*, const double*, double, int*,     \
                                   cudaStream_t);                                                \
  template void launch_set_damp<T>(const StepArgs<T>&, T*, const double*, double, int*, cudaStream_t); \
  template void launch_extract_owned<T>(const StepArgs<T>&, const T*, T*, cudaStream_t);              \
  template void launch_extract_face<T>(const StepArgs<T>&, const T*, int, T*, cudaStream_t);        \
  template void launch_refined_pair<T>(const StepArgs<T>&, cudaStream_t);

HYB_INSTANTIATE(float)
HYB_INSTANTIATE(double)

}  // namespace hyb
