// Time-step kernels of the hybrid FEM/FDM scheme.
//
// One launch advances every slot (source / problem) by one time level.  A
// thread owns one (x, y) column of the lattice and marches a chunk of z
// planes, keeping u at z-1, z, z+1 in registers; x/y neighbours come through
// L1.  Three row kinds share the launch:
//  * FDM rows, Eq. (fdmschemeforward): u^{k+1} = 2u^k - u^{k-1} + tau^2 Delta_h u^k,
//  * FEM rows on the FEM-owned nodes, Eq. (fem) with lumped mass: on the
//    Kuhn-cut voxels the row is a 7-point stencil whose axis-edge weight is
//    W = sum over the four voxels around the edge of a_c / 3 (edge touching
//    the voxel's diagonal corners) or a_c / 6,
//  * boundary rows: Neumann mirror ghosts, the plane-wave flux of Eq. (f),
//    and the absorbing rows of Eq. (eq:abs2), which use the new value of the
//    inward neighbour; a boundary thread recomputes that value itself, so no
//    intra-step synchronisation is needed.
// Both schemes write the same field, so the omega_o / omega_diamond copies
// of Algorithm 1 need no data movement.
//
// The adjoint kernel is the exact transpose of the forward step (the
// discrete form of Eq. (adjoint1)).  Away from the outer boundary the
// mass-weighted operator is symmetric, so the transposed row is the forward
// stencil; within one node of the boundary each node gathers the transposed
// coefficients of its neighbours' rows (mirror factors, absorbing rows) and
// solves the transposed absorbing coupling by recomputing the outer values.
// The same launch accumulates, per unknown voxel and in FP64, the sum over
// the voxel's 12 axis edges of w_e (u_p - u_q)(lambda_p - lambda_q) with
// w_e = 1/3 or 1/6; the host scales it by -tau^2 / h^2 (Eq. (gradient1)).
#include "hyb_internal.h"

namespace hyb {
namespace {

__device__ __forceinline__ int face_bits(int i, int j, int k, int nx, int ny, int nz) {
  return (i == 0 ? 1 : 0) | (i == nx - 1 ? 2 : 0) | (j == 0 ? 4 : 0) | (j == ny - 1 ? 8 : 0) |
         (k == 0 ? 16 : 0) | (k == nz - 1 ? 32 : 0);
}

template <typename T>
__device__ __forceinline__ long long lin(const StepArgs<T>& A, int i, int j, int k) {
  return (long long)i + (long long)A.nx * ((long long)j + (long long)A.ny * k);
}

template <typename T>
__device__ __forceinline__ bool fem_owned(const StepArgs<T>& A, int i, int j, int k) {
  return i >= A.fl[0] && i <= A.fh[0] && j >= A.fl[1] && j <= A.fh[1] && k >= A.fl[2] &&
         k <= A.fh[2];
}

template <typename T>
__device__ __forceinline__ long long widx(const StepArgs<T>& A, int i, int j, int k) {
  return (long long)(i - A.wl[0]) +
         (long long)A.wn[0] * ((long long)(j - A.wl[1]) + (long long)A.wn[1] * (k - A.wl[2]));
}

// sum over the six axis edges of W_e (u_nb - u_c) at a FEM-owned node
template <typename T>
__device__ __forceinline__ T fem_lap(const StepArgs<T>& A, const T* __restrict__ u, long long id,
                                     int i, int j, int k, T c, T zm, T zp) {
  const long long w = widx(A, i, j, k);
  const T* Wx = A.W;
  const T* Wy = A.W + A.wsz;
  const T* Wz = A.W + 2 * A.wsz;
  const long long wy = A.wn[0];
  const long long wz = (long long)A.wn[0] * A.wn[1];
  return Wx[w] * (u[id + 1] - c) + Wx[w - 1] * (u[id - 1] - c) + Wy[w] * (u[id + A.nx] - c) +
         Wy[w - wy] * (u[id - A.nx] - c) + Wz[w] * (zp - c) + Wz[w - wz] * (zm - c);
}

// Laplacian part (without 1/h^2) of a non-absorbing row at any node:
// FEM stencil on FEM-owned nodes, 7-point with mirror ghosts elsewhere.
template <typename T>
__device__ __noinline__ T row_lap(const StepArgs<T>& A, const T* __restrict__ u, int i, int j, int k) {
  const long long id = lin(A, i, j, k);
  const long long sz = (long long)A.nx * A.ny;
  const T c = u[id];
  if (fem_owned(A, i, j, k)) return fem_lap(A, u, id, i, j, k, c, u[id - sz], u[id + sz]);
  T lap = T(0);
  if (i == 0) lap += T(2) * (u[id + 1] - c);
  else if (i == A.nx - 1) lap += T(2) * (u[id - 1] - c);
  else lap += (u[id - 1] - c) + (u[id + 1] - c);
  if (j == 0) lap += T(2) * (u[id + A.nx] - c);
  else if (j == A.ny - 1) lap += T(2) * (u[id - A.nx] - c);
  else lap += (u[id - A.nx] - c) + (u[id + A.nx] - c);
  if (k == 0) lap += T(2) * (u[id + sz] - c);
  else if (k == A.nz - 1) lap += T(2) * (u[id - sz] - c);
  else lap += (u[id - sz] - c) + (u[id + sz] - c);
  return lap;
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
          acc += S.cur[lin(A, i1, j1, k1)] - A.r * fwd_new<T, D - 1>(A, S, i1, j1, k1);
        }
      }
      return A.r * S.cur[id] + acc / T(__popc(fb));
    }
  }
  T v = T(2) * S.cur[id] - S.prev[id] + A.c2 * row_lap(A, S.cur, i, j, k);
  if (S.src_face >= 0 && ((fall >> S.src_face) & 1)) v += S.srcval;
  return v;
}

// Coefficient of the non-absorbing row of node (i,j,k) on its neighbour
// (i,j,k) + s e_ax (Laplacian part, without 1/h^2).
template <typename T>
__device__ __forceinline__ T row_coef(const StepArgs<T>& A, int i, int j, int k, int ax, int s) {
  if (fem_owned(A, i, j, k)) {
    const long long w = widx(A, i, j, k);
    const long long ws = ax == 0 ? 1 : (ax == 1 ? (long long)A.wn[0] : (long long)A.wn[0] * A.wn[1]);
    return A.W[ax * A.wsz + (s > 0 ? w : w - ws)];
  }
  const int c = ax == 0 ? i : (ax == 1 ? j : k);
  const int n = ax == 0 ? A.nx : (ax == 1 ? A.ny : A.nz);
  if ((s > 0 && c == 0) || (s < 0 && c == n - 1)) return T(2);
  return T(1);
}

template <typename T>
__device__ __forceinline__ T row_diag(const StepArgs<T>& A, int i, int j, int k) {
  if (fem_owned(A, i, j, k)) {
    const long long w = widx(A, i, j, k);
    const long long wy = A.wn[0];
    const long long wz = (long long)A.wn[0] * A.wn[1];
    const T* W = A.W;
    return -(W[w] + W[w - 1] + W[A.wsz + w] + W[A.wsz + w - wy] + W[2 * A.wsz + w] +
             W[2 * A.wsz + w - wz]);
  }
  return T(-6);
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
  if (fbm & S.mask_f) rhs = A.r * l1[id];
  else rhs = (T(2) + A.c2 * row_diag(A, i, j, k)) * l1[id];
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
        rhs += A.c2 * row_coef(A, ni, nj, nk, ax, -s) * l1[nid];
      }
    }
  }
  if (!(fbm & S.mask_c)) rhs -= S.prev[id];
  if (S.obs_r && ((fbm >> S.obs_face) & 1)) rhs += S.obs_r[face_index(S.obs_face, i, j, k, A.nx, A.ny)];
  return rhs;
}

// lambda^j at node m: solve E_{j-1}^T lambda^j = rhs, where E couples an
// absorbing node b to its inward neighbours with r / L_b.
template <typename T, int D>
__device__ __noinline__ T adj_new(const StepArgs<T>& A, const Slot<T>& S, int i, int j, int k) {
  T v = adj_rhs(A, S, i, j, k);
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
        if (fbb & (1 << f)) v -= (A.r / T(__popc(fbb))) * adj_new<T, D - 1>(A, S, bi, bj, bk);
      }
    }
  }
  return v;
}

// sum over the 12 axis edges of voxel (i,j,k) of w_e (u_p - u_q)(l_p - l_q)
template <typename T>
__device__ __forceinline__ T voxel_pair(const StepArgs<T>& A, const T* __restrict__ hb,
                                        const T* __restrict__ lam, int i, int j, int k) {
  const long long hy = A.fn[0];
  const long long hz = (long long)A.fn[0] * A.fn[1];
  const long long h0 = (long long)(i - A.fl[0]) + hy * (j - A.fl[1]) + hz * (k - A.fl[2]);
  const long long ly = A.nx;
  const long long lz = (long long)A.nx * A.ny;
  const long long l0 = lin(A, i, j, k);
  T u[8], l[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int a = c & 1, b = (c >> 1) & 1, d = c >> 2;
    u[c] = hb[h0 + a + b * hy + d * hz];
    l[c] = lam[l0 + a + b * ly + d * lz];
  }
  const T d3 = (u[1] - u[0]) * (l[1] - l[0]) + (u[7] - u[6]) * (l[7] - l[6]) +
               (u[2] - u[0]) * (l[2] - l[0]) + (u[7] - u[5]) * (l[7] - l[5]) +
               (u[4] - u[0]) * (l[4] - l[0]) + (u[7] - u[3]) * (l[7] - l[3]);
  const T d6 = (u[3] - u[2]) * (l[3] - l[2]) + (u[5] - u[4]) * (l[5] - l[4]) +
               (u[3] - u[1]) * (l[3] - l[1]) + (u[6] - u[4]) * (l[6] - l[4]) +
               (u[5] - u[1]) * (l[5] - l[1]) + (u[6] - u[2]) * (l[6] - l[2]);
  return d3 / T(3) + d6 / T(6);
}

// Node t of the boundary shell of thickness TH (every node with a coordinate
// closer than TH to a face), enumerated as whole z planes, then whole y rows
// of the remaining planes, then the x ends of the remaining rows.
template <typename T, int TH>
__device__ __forceinline__ void shell_node(const StepArgs<T>& A, long long t, int& i, int& j, int& k) {
  const int nx = A.nx, ny = A.ny, nz = A.nz;
  const int ix = max(nx - 2 * TH, 0), iy = max(ny - 2 * TH, 0), iz = max(nz - 2 * TH, 0);
  const long long plane = (long long)nx * ny;
  const long long na = (long long)(nz - iz) * plane;
  if (t < na) {
    const int p = (int)(t / plane);
    const long long r = t - (long long)p * plane;
    k = p < TH ? p : p + iz;
    j = (int)(r / nx);
    i = (int)(r - (long long)j * nx);
    return;
  }
  t -= na;
  const long long rowsz = (long long)(ny - iy) * nx;
  const long long nb = (long long)iz * rowsz;
  if (t < nb) {
    const int pk = (int)(t / rowsz);
    const long long r = t - (long long)pk * rowsz;
    k = TH + pk;
    const int row = (int)(r / nx);
    j = row < TH ? row : row + iy;
    i = (int)(r - (long long)row * nx);
    return;
  }
  t -= nb;
  const int w = nx - ix;
  const long long idx = t / w;
  const int c = (int)(t - idx * w);
  k = TH + (int)(idx / iy);
  j = TH + (int)(idx % iy);
  i = c < TH ? c : c + ix;
}

template <typename T>
__device__ __forceinline__ void pair_if_voxel(const StepArgs<T>& A, const Slot<T>& S, int si, int i, int j,
                                              int k) {
  if (S.hist_r == nullptr) return;
  if (i < A.fl[0] || i >= A.fl[0] + A.un[0] || j < A.fl[1] || j >= A.fl[1] + A.un[1] || k < A.fl[2] ||
      k >= A.fl[2] + A.un[2])
    return;
  const long long nv = (long long)A.un[0] * A.un[1] * A.un[2];
  const long long vid = (long long)(i - A.fl[0]) +
                        (long long)A.un[0] * ((j - A.fl[1]) + (long long)A.un[1] * (k - A.fl[2]));
  A.G[(long long)si * nv + vid] += (double)voxel_pair(A, S.hist_r, S.cur, i, j, k);
}

// Laplacian part of the row of a node that lies on no face (all six
// neighbours exist, no mirror): FEM stencil or 7-point FDM.
template <typename T>
__device__ __forceinline__ T interior_lap(const StepArgs<T>& A, const T* __restrict__ u, long long id, int i,
                                          int j, int k) {
  const long long pl = (long long)A.nx * A.ny;
  const T c = u[id];
  if (fem_owned(A, i, j, k)) return fem_lap(A, u, id, i, j, k, c, u[id - pl], u[id + pl]);
  return (u[id - 1] - c) + (u[id + 1] - c) + (u[id - A.nx] - c) + (u[id + A.nx] - c) + (u[id - pl] - c) +
         (u[id + pl] - c);
}

template <typename T>
__device__ __forceinline__ long long axis_stride(const StepArgs<T>& A, int ax) {
  return ax == 0 ? 1LL : (ax == 1 ? (long long)A.nx : (long long)A.nx * A.ny);
}

// Interior kernel shared by the forward (TH = 1) and adjoint (TH = 2)
// steps: 32 x 8 thread tiles of the interior box, each thread marching a
// chunk of z planes with u at z-1, z, z+1 in registers and the next plane
// and the previous-level value loaded one iteration ahead.
template <typename T, int TH, bool ADJ>
__global__ void __launch_bounds__(kTileX * kTileY) bulk_kernel(const __grid_constant__ StepArgs<T> A) {
  const int tps = A.npb * A.nzc;
  const int si = blockIdx.x / tps;
  int rem = blockIdx.x - si * tps;
  const int zc = rem / A.npb;
  rem -= zc * A.npb;
  const int tyy = rem / A.ntx;
  const int txx = rem - tyy * A.ntx;
  const int nx = A.nx, ny = A.ny, nz = A.nz;
  const int i = TH + txx * kTileX + (threadIdx.x % kTileX);
  const int j = TH + tyy * kTileY + (threadIdx.x / kTileX);
  if (i > nx - 1 - TH || j > ny - 1 - TH) return;
  const int z0 = TH + zc * A.zchunk;
  const int z1 = min(z0 + A.zchunk, nz - TH);
  if (z0 >= z1) return;
  const Slot<T>& S = A.s[si];
  const long long plane = (long long)nx * ny;
  const T* __restrict__ c = S.cur;
  const T* __restrict__ p = S.prev;
  T* __restrict__ out = S.next;
  const bool xy_fem = i >= A.fl[0] && i <= A.fh[0] && j >= A.fl[1] && j <= A.fh[1];
  const bool xy_vox = ADJ && S.hist_r != nullptr && i >= A.fl[0] && i < A.fl[0] + A.un[0] &&
                      j >= A.fl[1] && j < A.fl[1] + A.un[1];
  T* __restrict__ hw = ADJ ? nullptr : S.hist_w;
  const long long nv = (long long)A.un[0] * A.un[1] * A.un[2];
  long long id = (long long)i + (long long)nx * j + plane * z0;
  T cm = c[id - plane];
  T c0 = c[id];
  T cp = c[id + plane];
  T pv = p[id];
  const T c2 = A.c2;
  for (int k = z0; k < z1; ++k, id += plane) {
    const T cpp = (k + 2 <= nz - 1) ? c[id + 2 * plane] : T(0);
    const T pvn = (k + 1 < z1) ? p[id + plane] : T(0);
    T val;
    const bool fem = xy_fem && k >= A.fl[2] && k <= A.fh[2];
    if (fem) {
      val = T(2) * c0 - pv + c2 * fem_lap(A, c, id, i, j, k, c0, cm, cp);
      if (hw)
        hw[(long long)(i - A.fl[0]) + (long long)A.fn[0] * ((j - A.fl[1]) + (long long)A.fn[1] * (k - A.fl[2]))] =
            val;
    } else {
      const T lap = (c[id - 1] - c0) + (c[id + 1] - c0) + (c[id - nx] - c0) + (c[id + nx] - c0) + (cm - c0) +
                    (cp - c0);
      val = T(2) * c0 - pv + c2 * lap;
    }
    out[id] = val;
    if (ADJ && xy_vox && k >= A.fl[2] && k < A.fl[2] + A.un[2]) {
      const long long vid = (long long)(i - A.fl[0]) +
                            (long long)A.un[0] * ((j - A.fl[1]) + (long long)A.un[1] * (k - A.fl[2]));
      A.G[(long long)si * nv + vid] += (double)voxel_pair(A, S.hist_r, c, i, j, k);
    }
    cm = c0;
    c0 = cp;
    cp = cpp;
    pv = pvn;
  }
}

// Outer faces: Neumann, source and absorbing rows; trace record.  A node on
// a single face takes an inlined row; edge and corner nodes the generic one.
template <typename T>
__global__ void __launch_bounds__(128) fwd_shell_kernel(const __grid_constant__ StepArgs<T> A) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long ns = A.nshell;
  if (t >= ns * A.nslots) return;
  const int si = (int)(t / ns);
  int i, j, k;
  shell_node<T, 1>(A, t - (long long)si * ns, i, j, k);
  const Slot<T>& S = A.s[si];
  const int fall = face_bits(i, j, k, A.nx, A.ny, A.nz);
  const long long id = lin(A, i, j, k);
  T val;
  if (__popc(fall) == 1) {
    const int f = __ffs(fall) - 1;
    const int ax = f >> 1;
    const int step = (f & 1) ? -1 : 1;  // inward
    const long long sa = axis_stride(A, ax);
    const T* __restrict__ u = S.cur;
    const T* __restrict__ up = S.prev;
    if (S.mask_f & fall) {
      // Eq. (eq:abs2) with the new value of the inward neighbour b1
      const long long id1 = id + step * sa;
      const T n1 = T(2) * u[id1] - up[id1] +
                   A.c2 * interior_lap(A, u, id1, i + (ax == 0 ? step : 0), j + (ax == 1 ? step : 0),
                                       k + (ax == 2 ? step : 0));
      val = A.r * u[id] + (u[id1] - A.r * n1);
    } else {
      // mirror ghost along the face normal, plus the source flux
      const T cc = u[id];
      T lap = T(2) * (u[id + step * sa] - cc);
#pragma unroll
      for (int a2 = 0; a2 < 3; ++a2) {
        if (a2 == ax) continue;
        const long long s2 = axis_stride(A, a2);
        lap += (u[id - s2] - cc) + (u[id + s2] - cc);
      }
      val = T(2) * cc - up[id] + A.c2 * lap;
      if (S.src_face == f) val += S.srcval;
    }
  } else {
    val = fwd_new<T, 3>(A, S, i, j, k);
  }
  S.next[id] = val;
  if (S.obs_w && ((fall >> S.obs_face) & 1)) S.obs_w[face_index(S.obs_face, i, j, k, A.nx, A.ny)] = val;
}

// lambda^j at a node on the single face f whose in-face coordinates are at
// least two nodes from the other faces (no transposed absorbing coupling
// reaches it).
template <typename T>
__device__ __forceinline__ T adj_face_interior(const StepArgs<T>& A, const Slot<T>& S, int i, int j, int k,
                                               int f) {
  const T* __restrict__ l1 = S.cur;
  const long long id = lin(A, i, j, k);
  const int ax = f >> 1;
  const int step = (f & 1) ? -1 : 1;
  const long long sa = axis_stride(A, ax);
  const bool abc = (S.mask_f >> f) & 1;
  T rhs = abc ? A.r * l1[id] : (T(2) - T(6) * A.c2) * l1[id];
  rhs += A.c2 *
         row_coef(A, i + (ax == 0 ? step : 0), j + (ax == 1 ? step : 0), k + (ax == 2 ? step : 0), ax, -step) *
         l1[id + step * sa];
  if (!abc) {
#pragma unroll
    for (int a2 = 0; a2 < 3; ++a2) {
      if (a2 == ax) continue;
      const long long s2 = axis_stride(A, a2);
      rhs += A.c2 * (l1[id - s2] + l1[id + s2]);
    }
  }
  if (!((S.mask_c >> f) & 1)) rhs -= S.prev[id];
  if (S.obs_r && S.obs_face == f) rhs += S.obs_r[face_index(f, i, j, k, A.nx, A.ny)];
  return rhs;
}

// Nodes within one node of a face.  Inlined rows for the two common cases
// (on one face, or one node inside one face, away from edges); the generic
// transposed gather for the rest.
template <typename T>
__global__ void __launch_bounds__(128) adj_shell_kernel(const __grid_constant__ StepArgs<T> A) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long ns = A.nshell;
  if (t >= ns * A.nslots) return;
  const int si = (int)(t / ns);
  int i, j, k;
  shell_node<T, 2>(A, t - (long long)si * ns, i, j, k);
  const Slot<T>& S = A.s[si];
  const int cc[3] = {i, j, k};
  const int nn[3] = {A.nx, A.ny, A.nz};
  int n0 = 0, n1 = 0, a0 = 0, a1 = 0;
  bool fast = nn[0] >= 4 && nn[1] >= 4 && nn[2] >= 4;
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    const int d = min(cc[ax], nn[ax] - 1 - cc[ax]);
    if (d == 0) {
      ++n0;
      a0 = ax;
    } else if (d == 1) {
      ++n1;
      a1 = ax;
    }
  }
  const long long id = lin(A, i, j, k);
  T val;
  if (fast && n0 == 1 && n1 == 0) {
    val = adj_face_interior(A, S, i, j, k, 2 * a0 + (cc[a0] == 0 ? 0 : 1));
  } else if (fast && n0 == 0 && n1 == 1) {
    // one node inside face f; b is the face node next to it
    const int f = 2 * a1 + (cc[a1] == 1 ? 0 : 1);
    const int bs = (f & 1) ? 1 : -1;  // from m towards b
    const T* __restrict__ l1 = S.cur;
    T rhs = (T(2) + A.c2 * row_diag(A, i, j, k)) * l1[id];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
#pragma unroll
      for (int tt = 0; tt < 2; ++tt) {
        const int s = tt ? 1 : -1;
        const long long nid = id + s * axis_stride(A, ax);
        if (ax == a1 && s == bs) {
          rhs += ((S.mask_f >> f) & 1) ? l1[nid] : T(2) * A.c2 * l1[nid];
        } else {
          rhs += A.c2 *
                 row_coef(A, i + (ax == 0 ? s : 0), j + (ax == 1 ? s : 0), k + (ax == 2 ? s : 0), ax, -s) *
                 l1[nid];
        }
      }
    }
    rhs -= S.prev[id];
    if ((S.mask_e >> f) & 1) {
      rhs -= A.r * adj_face_interior(A, S, i + (a1 == 0 ? bs : 0), j + (a1 == 1 ? bs : 0),
                                     k + (a1 == 2 ? bs : 0), f);
    }
    val = rhs;
  } else {
    val = adj_new<T, 3>(A, S, i, j, k);
  }
  S.next[id] = val;
  pair_if_voxel(A, S, si, i, j, k);
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
  grad[t] += (double)voxel_pair(A, hist, lam, A.fl[0] + x, A.fl[1] + y, A.fl[2] + z);
}

template <typename T>
__global__ void set_coef_kernel(const __grid_constant__ StepArgs<T> A, T* __restrict__ W,
                                const double* __restrict__ a, double a_max, int* flag) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nv = (long long)A.un[0] * A.un[1] * A.un[2];
  if (t < nv) {
    const double v = a[t];
    if (!(v <= a_max * (1.0 + 1e-12)) || !(v == v)) atomicExch(flag, 1);
  }
  if (t >= A.wsz) return;
  const int p[3] = {A.wl[0] + (int)(t % A.wn[0]), A.wl[1] + (int)((t / A.wn[0]) % A.wn[1]),
                    A.wl[2] + (int)(t / ((long long)A.wn[0] * A.wn[1]))};
  for (int ax = 0; ax < 3; ++ax) {
    double w = 0.0;
    if (p[ax] + 1 <= A.wl[ax] + A.wn[ax] - 1) {
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
    W[ax * A.wsz + t] = (T)w;
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
  box[t] = f[lin(A, A.fl[0] + x, A.fl[1] + y, A.fl[2] + z)];
}

}  // namespace

template <typename T>
void launch_forward(const StepArgs<T>& a, cudaStream_t st) {
  const unsigned grid = (unsigned)(a.npb * a.nzc * a.nslots);
  if (grid) bulk_kernel<T, 1, false><<<grid, kTileX * kTileY, 0, st>>>(a);
  const long long n = a.nshell * a.nslots;
  fwd_shell_kernel<T><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(a);
}

template <typename T>
void launch_adjoint(const StepArgs<T>& a, cudaStream_t st) {
  const unsigned grid = (unsigned)(a.npb * a.nzc * a.nslots);
  if (grid) bulk_kernel<T, 2, true><<<grid, kTileX * kTileY, 0, st>>>(a);
  const long long n = a.nshell * a.nslots;
  adj_shell_kernel<T><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(a);
}

template <typename T>
void launch_pair(const StepArgs<T>& a, const T* hist, const T* lam, cudaStream_t st) {
  const long long nv = (long long)a.un[0] * a.un[1] * a.un[2];
  if (nv == 0) return;
  pair_kernel<T><<<(unsigned)((nv + 255) / 256), 256, 0, st>>>(a, hist, lam, a.G);
}

template <typename T>
void launch_set_coef(const StepArgs<T>& a, T* W, const double* acoef, double a_max, int* flag,
                     cudaStream_t st) {
  const long long nv = (long long)a.un[0] * a.un[1] * a.un[2];
  const long long n = a.wsz > nv ? a.wsz : nv;
  if (n == 0) return;
  set_coef_kernel<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, W, acoef, a_max, flag);
}

template <typename T>
void launch_extract_owned(const StepArgs<T>& a, const T* field, T* box, cudaStream_t st) {
  const long long n = (long long)a.fn[0] * a.fn[1] * a.fn[2];
  if (n == 0) return;
  extract_owned_kernel<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, field, box);
}

#define HYB_INSTANTIATE(T)                                                                       \
  template void launch_forward<T>(const StepArgs<T>&, cudaStream_t);                             \
  template void launch_adjoint<T>(const StepArgs<T>&, cudaStream_t);                             \
  template void launch_pair<T>(const StepArgs<T>&, const T*, const T*, cudaStream_t);            \
  template void launch_set_coef<T>(const StepArgs<T>&, T*, const double*, double, int*,         \
                                   cudaStream_t);                                                \
  template void launch_extract_owned<T>(const StepArgs<T>&, const T*, T*, cudaStream_t);

HYB_INSTANTIATE(float)
HYB_INSTANTIATE(double)

}  // namespace hyb
