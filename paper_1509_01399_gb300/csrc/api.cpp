// Host side of the C ABI declared in include/hyb.h: argument checking,
// device workspaces, the time loops of Algorithm 2 (forward, and backward in
// time for the adjoint with optional checkpoint/recompute), the gradient of
// Eq. (gradient1) and one iteration of Algorithm 3.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <array>
#include <utility>
#include <vector>

#include "hyb_internal.h"

using namespace hyb;

namespace {

thread_local std::string g_err;

hyb_status fail(hyb_status st, const char* fmt, ...) {
  char buf[768];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

// Identity of one sweep's launch sequence: everything baked into the kernel
// parameters of a captured CUDA graph.
struct SweepKey {
  int kind = -1;  // 0 forward keeping history, 1 forward without, 2 adjoint
  int batch = 0;  // per-slot coefficients
  const void* io = nullptr;
  int accumulate = 0;
  int nsteps = 0, nsrc = 0;
  double dt = 0.0;
  int face[16] = {0};
  double omega[16] = {0.0}, amp[16] = {0.0}, dir[16][3] = {};
  const void* bufs[10] = {nullptr};
};

bool same_key(const SweepKey& a, const SweepKey& b) {
  if (a.kind != b.kind || a.batch != b.batch || a.io != b.io || a.accumulate != b.accumulate || a.nsteps != b.nsteps ||
      a.nsrc != b.nsrc || a.dt != b.dt)
    return false;
  for (int i = 0; i < a.nsrc; ++i)
    if (a.face[i] != b.face[i] || a.omega[i] != b.omega[i] || a.amp[i] != b.amp[i] || a.dir[i][0] != b.dir[i][0] ||
        a.dir[i][1] != b.dir[i][1] || a.dir[i][2] != b.dir[i][2])
      return false;
  for (int i = 0; i < 10; ++i)
    if (a.bufs[i] != b.bufs[i]) return false;
  return true;
}

// A sweep is captured into a graph the second time the same key is seen and
// replayed while the key stays the same.
struct SweepGraph {
  SweepKey key, last;
  bool seen = false;
  cudaGraphExec_t exec = nullptr;
  long long launches = 0;
};

}  // namespace

struct hyb_mesh {
  hyb_mesh_desc d;
  cudaStream_t st = nullptr;
  int n[3] = {0, 0, 0};
  long long N = 0;    // lattice nodes
  int px = 0;         // row pitch of the lattice fields (multiple of 8)
  long long Np = 0;   // entries of one lattice field (px ny nz)
  bool fem = false;
  int fl[3], fh[3], fn[3], wl[3], wn[3], un[3];
  int wx0 = 0, wpx = 0;  // edge-weight arrays: x origin and row pitch (multiples of 4)
  int hx0 = 0, hpx = 0;  // FEM-owned (history) box: x origin and row pitch (multiples of 8)
  long long wsz = 0, nu = 0, nown = 0;
  long long hbox = 0;    // entries of one history box (hpx fn1 fn2)
  int obs_stride = 0;
  int abc_mask = 0;
  DevBuf W, G, flag, U, L, hist, ckpt, part, scal, g, atrial, cot, trace;
  double* hscal = nullptr;  // pinned host copy of device scalars
  bool have_fwd = false;    // the adjoint has what it needs
  bool have_run = false;    // a forward has run (time grid known)
  bool have_adj = false;
  bool u_levels = false;    // U still holds the last forward's final levels
  bool batch = false;       // the last forward gave every slot its own coefficient
  int nsteps = 0, nsrc = 0;
  double dt = 0.0;
  hyb_source src[kMaxSlots];
  long long launches = 0;
  long long bytes = 0;
  // refined region
  int nc = 0, nr = 0, nrl = 0, nnz = 0;
  double dt_max = 0.0;
  DevBuf rmask, rzr, refvox, refvox_id, k9, rcid, avox, rpos, rvxyz;
  DevBuf sdamp, ones;  // telegraph model: damping ratios (history-box layout), a = 1 on the unknown voxels
  double uK9[81], uK8[64], um9[9], um8[8];  // unit-voxel stiffness and lumped masses (refined, Kuhn)
  DevBuf CU, CL, chist, cckpt;  // centre values (levels, history, checkpoints)
  DevBuf I0, IC0;               // initial state of Model Problem 1: u^0, u^{-1} (padded fields), centres
  DevBuf acopy, kuhn, kuhn_v;   // all-FEM path: coefficient of the last forward, Kuhn element tables
  bool have_init = false;
  bool ani = false;          // the lattice steps differ per axis (every level by the bulk and shell kernels)
  double hv[3] = {0, 0, 0};  // lattice step per axis
  cudaStream_t cap = nullptr;  // private stream used only to capture sweep graphs
  // interior work items of the forward / transposed step per slot count; built
  // once and kept (captured sweep graphs refer to them)
  DevBuf items[2][kMaxSlots + 1];
  int nitems[2][kMaxSlots + 1] = {};
  int nsm = 0;                 // SMs of the device
  int bps = 0;                 // resident step-kernel blocks per SM
  SweepGraph graphs[3];
};

#define HYB_CU(call)                                                                      \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) return fail(HYB_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

#define HYB_LAUNCHED(m)                                                                  \
  do {                                                                                   \
    ++(m)->launches;                                                                     \
    cudaError_t e_ = cudaGetLastError();                                                 \
    if (e_ != cudaSuccess) return fail(HYB_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(e_)); \
  } while (0)

#define HYB_TRY(expr)                 \
  do {                                \
    hyb_status s_ = (expr);           \
    if (s_ != HYB_OK) return s_;      \
  } while (0)

namespace {

hyb_status ensure(hyb_mesh* m, DevBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return HYB_OK;
  if (b.p) {
    cudaError_t e = cudaStreamSynchronize(m->st);
    if (e != cudaSuccess) return fail(HYB_ERR_CUDA, "sync before realloc: %s", cudaGetErrorString(e));
    cudaFree(b.p);
    m->bytes -= (long long)b.bytes;
    b.p = nullptr;
    b.bytes = 0;
  }
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    return fail(HYB_ERR_OOM, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
  }
  b.bytes = bytes;
  m->bytes += (long long)bytes;
  return HYB_OK;
}

void release(DevBuf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

size_t esize(const hyb_mesh* m) { return m->d.precision == HYB_FP64 ? 8 : 4; }

SweepKey make_key(const hyb_mesh* m, int kind, const void* io, int accumulate, int nsteps, int nsrc, double dt,
                  const hyb_source* src) {
  SweepKey k;
  k.kind = kind;
  k.batch = m->batch ? 1 : 0;
  k.io = io;
  k.accumulate = accumulate;
  k.nsteps = nsteps;
  k.nsrc = nsrc;
  k.dt = dt;
  for (int i = 0; i < nsrc; ++i) {
    k.face[i] = src[i].face;
    k.omega[i] = src[i].omega;
    k.amp[i] = src[i].amp;
    for (int a = 0; a < 3; ++a) k.dir[i][a] = src[i].dir[a];
  }
  const void* b[10] = {m->U.p, m->L.p, m->hist.p, m->ckpt.p, m->G.p, m->W.p, m->CU.p, m->CL.p,
                       m->have_init ? m->I0.p : nullptr, m->have_init ? m->IC0.p : nullptr};
  for (int i = 0; i < 10; ++i) k.bufs[i] = b[i];
  return k;
}

// Run a sweep body (memsets, copies and step launches on the given stream):
// replay its graph when the key matches the captured one, capture it on the
// second call with the same key, run it directly otherwise.  Bodies must not
// allocate or synchronise.
template <class Body>
hyb_status run_sweep(hyb_mesh* m, SweepGraph& g, const SweepKey& key, Body body) {
  if (g.exec && same_key(g.key, key)) {
    HYB_CU(cudaGraphLaunch(g.exec, m->st));
    m->launches += g.launches;
    return HYB_OK;
  }
  const bool capture = g.seen && same_key(g.last, key);
  g.last = key;
  g.seen = true;
  if (!capture) return body(m->st);
  if (g.exec) {
    cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
  }
  if (cudaStreamBeginCapture(m->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return body(m->st);
  }
  const long long l0 = m->launches;
  const hyb_status st = body(m->cap);
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(m->cap, &graph);
  const long long n = m->launches - l0;
  m->launches = l0;
  if (st != HYB_OK || e != cudaSuccess || !graph) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    if (st != HYB_OK) return st;
    return body(m->st);
  }
  const cudaError_t ei = cudaGraphInstantiate(&g.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) {
    cudaGetLastError();
    g.exec = nullptr;
    return body(m->st);
  }
  g.key = key;
  g.launches = n;
  HYB_CU(cudaGraphLaunch(g.exec, m->st));
  m->launches += n;
  return HYB_OK;
}

// Plane wave launched by a source (Eq. (f) at normal or oblique incidence):
// unit direction d (d = -n of the face for a face source), entry corner i0
// (the box corner where d . x is smallest), the factor -(d . n_f) of the flux
// on each entry face (0 on the others) and the last instant each entry face
// carries it: t1 plus the largest delay d . (x - x0) over the face.
struct Wave {
  double d[3];
  int i0[3];
  double fac[6];
  double tsw[6];
};

Wave wave_of(const hyb_mesh* m, const hyb_source& s) {
  Wave w;
  double d[3] = {s.dir[0], s.dir[1], s.dir[2]};
  if (d[0] == 0.0 && d[1] == 0.0 && d[2] == 0.0) {
    const int ax = s.face >> 1;
    d[ax] = (s.face & 1) ? -1.0 : 1.0;
  }
  const double nrm = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  for (int a = 0; a < 3; ++a) {
    w.d[a] = d[a] / nrm;
    w.i0[a] = w.d[a] >= 0.0 ? 0 : m->n[a] - 1;
  }
  const double t1 = 2.0 * M_PI / s.omega;
  for (int f = 0; f < 6; ++f) {
    const int ax = f >> 1;
    const double dn = w.d[ax] * ((f & 1) ? 1.0 : -1.0);
    w.fac[f] = dn < 0.0 ? -dn : 0.0;
    const int p = ax == 0 ? 1 : 0, q = ax == 2 ? 1 : 2;
    if (m->ani)
      w.tsw[f] = t1 + (std::fabs(w.d[p]) * (m->n[p] - 1) * m->hv[p] + std::fabs(w.d[q]) * (m->n[q] - 1) * m->hv[q]);
    else
      w.tsw[f] = t1 + m->d.h * (std::fabs(w.d[p]) * (m->n[p] - 1) + std::fabs(w.d[q]) * (m->n[q] - 1));
  }
  return w;
}

// Boundary state of the step leaving t_k = k dt for one source: an entry
// face carries the plane-wave flux while t_k <= its switch time (Model
// Problem 2: S_{1,1}, then S_{1,2}) and otherwise takes the mesh's own
// condition.  mask: absorbing faces; srcmask: faces carrying the flux.
void phase_of(const hyb_mesh* m, const hyb_source& s, int k, double dt, int* mask, int* srcmask) {
  const Wave w = wave_of(m, s);
  const double t = k * dt;
  int sm = 0;
  for (int f = 0; f < 6; ++f)
    if (w.fac[f] > 0.0 && t <= w.tsw[f]) sm |= 1 << f;
  *srcmask = sm;
  *mask = m->abc_mask & ~sm;
}

int mask_at(const hyb_mesh* m, const hyb_source& s, int k, double dt) {
  int mask, sm;
  phase_of(m, s, k, dt, &mask, &sm);
  return mask;
}

// The slot's plane-wave constants for the step leaving t_k.
template <typename T>
void set_wave(const hyb_mesh* m, Slot<T>& S, const hyb_source& src, int k, double dt) {
  const Wave w = wave_of(m, src);
  int mask, sm;
  phase_of(m, src, k, dt, &mask, &sm);
  S.mask_f = mask;
  S.src_mask = sm;
  S.st = k * dt;
  const double h = m->d.h;
  for (int f = 0; f < 6; ++f) S.sf[f] = dt * dt * 2.0 / (m->ani ? m->hv[f >> 1] : h) * src.amp * w.fac[f];
  for (int a = 0; a < 3; ++a) {
    S.sd[a] = m->ani ? w.d[a] * m->hv[a] : w.d[a];  // per-axis steps: the delay d . (x - x0) axis by axis
    S.si0[a] = w.i0[a];
  }
  S.sh = m->ani ? 1.0 : h;
  S.somega = src.omega;
  S.st1 = 2.0 * M_PI / src.omega;
}

// Launch geometry of one step: the interior covers nodes 1 .. n-2 on every
// axis in 32 x 16 tiles (in x from tile_x0: FP32 tiles start at x = 0); the edge tiles cover the nodes within one node of
// two faces.  Lattices with fewer than 5 nodes on an axis use a single
// generic kernel instead.
void step_geometry(const hyb_mesh* m, int* npb, int* ntx, int* small, int* nedge) {
  *small = (m->n[0] < 5 || m->n[1] < 5 || m->n[2] < 5) ? 1 : 0;
  *nedge = *small ? 0 : 1 + (m->n[0] - 4 + 7) / 8 + (m->n[1] - 4 + 7) / 8 + (m->n[2] - 4 + 7) / 8;
  *ntx = (m->n[0] - 1 - tile_x0(m->d.precision) + kTileX - 1) / kTileX;
  const int nty = (m->n[1] - 2 + kTileY - 1) / kTileY;
  *npb = *ntx * nty;
}

// Waves of resident interior blocks the work items are cut for: one when
// each resident block would get few tile levels (a block's first level waits
// for its planes, so long items pay off; two waves were 1-2 % faster for a
// lone sweep but cost a sixth of the throughput with several sweeps sharing
// the GPU), three when there is much work (blocks of uneven speed then even
// out within each SM).
constexpr int kStepWavesFew = 1, kStepWavesMany = 3;
constexpr double kManyLevelsPerBlock = 40.0;
constexpr double kZFaceLevelCost = 3.5;

// Interior work items of one step launch, one per block: (slot, tile, z0,
// z1).  Each tile's z range 1 .. n-2 is cut into pieces of about equal
// estimated cost, so that the items fill the chosen number of waves of the
// kernel's resident blocks evenly.  Relative cost of one tile level, fitted
// to per-block cycle counts on a 129^3 lattice (forward / transposed step),
// then adjusted by timing whole levels: 1 for a plain tile; 1.50
// / 1.70 for a tile next to an x or y face; 1.22 / 1.40 for a tile meeting
// the FEM block, plus 0.88 / 2.10 on planes where it holds FEM-owned nodes;
// plus kZFaceLevelCost on the two planes next to the z faces (they also
// produce the face plane and, on the source face, the trace).
std::vector<int> build_items(const hyb_mesh* m, int nslots, bool adjoint) {
  const int nx = m->n[0], ny = m->n[1], nz = m->n[2];
  const int x0 = tile_x0(m->d.precision);
  const int ntx = (nx - 1 - x0 + kTileX - 1) / kTileX, nty = (ny - 2 + kTileY - 1) / kTileY;
  struct Tile {
    int si, tile;
    double base, extra;
  };
  std::vector<Tile> tiles;
  double total = 0.0;
  const int zf0 = m->fl[2], zf1 = m->fh[2];
  const int fem_levels = m->fem ? std::max(0, std::min(zf1, nz - 2) - std::max(zf0, 1) + 1) : 0;
  for (int si = 0; si < nslots; ++si)
    for (int ty = 0; ty < nty; ++ty)
      for (int tx = 0; tx < ntx; ++tx) {
        const int i0 = x0 + tx * kTileX, j0 = 1 + ty * kTileY;
        const bool face = i0 <= 1 || i0 + kTileX - 1 >= nx - 2 || j0 == 1 || j0 + kTileY - 1 >= ny - 2;
        const bool femt = m->fem && i0 <= m->fh[0] && i0 + kTileX - 1 >= m->fl[0] && j0 <= m->fh[1] &&
                          j0 + kTileY - 1 >= m->fl[1];
        const double base = face ? (adjoint ? 1.70 : 1.50) : (femt ? (adjoint ? 1.40 : 1.22) : 1.0);
        const Tile t{si, ty * ntx + tx, base, femt ? (adjoint ? 2.10 : 0.88) : 0.0};
        tiles.push_back(t);
        total += t.base * (nz - 2) + t.extra * fem_levels + 2 * kZFaceLevelCost;
      }
  const double resident = (double)std::max(m->nsm, 1) * std::max(m->bps, 1);
  const double levels_per_block = (double)tiles.size() * (nz - 2) / resident;
  const double cap = resident * (levels_per_block > kManyLevelsPerBlock ? kStepWavesMany : kStepWavesFew);
  const double target = total / cap;
  std::vector<std::pair<double, std::array<int, 4>>> items;
  for (const Tile& t : tiles) {
    double acc = 0.0;
    int z0 = 1;
    for (int k = 1; k <= nz - 2; ++k) {
      acc += t.base + ((k >= zf0 && k <= zf1) ? t.extra : 0.0) + ((k == 1 || k == nz - 2) ? kZFaceLevelCost : 0.0);
      if (acc >= target || k == nz - 2) {
        items.push_back({acc, {t.si, t.tile, z0, k + 1}});
        z0 = k + 1;
        acc = 0.0;
      }
    }
  }
  // by source, then by z slab, then by tile: the items of one source run
  // together, and the blocks resident at one time cover one slab of
  // neighbouring tiles, whose halo columns and slab-boundary planes they then
  // share in L2
  std::stable_sort(items.begin(), items.end(), [](const auto& a, const auto& b) {
    if (a.second[0] != b.second[0]) return a.second[0] < b.second[0];
    if (a.second[2] != b.second[2]) return a.second[2] < b.second[2];
    return a.second[1] < b.second[1];
  });
  std::vector<int> out;
  out.reserve(items.size() * 4);
  for (const auto& it : items) out.insert(out.end(), it.second.begin(), it.second.end());
  return out;
}

// One time level on `st`: one launch (two with per-axis steps).
template <class Launch>
hyb_status step_launch(hyb_mesh* m, cudaStream_t st, Launch launch) {
  const int n = launch(st);  // kernels the level took (two with per-axis steps)
  m->launches += n - 1;
  HYB_LAUNCHED(m);
  return HYB_OK;
}

// P1 element of a tetrahedron (vertex coordinates X[4][3]): volume and
// stiffness K_ij = |K| grad phi_i . grad phi_j (Sec. 7.2), a = 1.
void p1_tet(const double X[4][3], double* vol, double K[4][4]) {
  double J[3][3];
  for (int c = 0; c < 3; ++c)
    for (int r = 0; r < 3; ++r) J[r][c] = X[c + 1][r] - X[0][r];
  const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                     J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                     J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  double inv[3][3];  // inverse of J: row i = grad of the barycentric function of vertex i + 1
  inv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
  inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
  inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
  inv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
  inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
  inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
  inv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
  inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
  inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
  double g[4][3];
  for (int d = 0; d < 3; ++d) {
    g[1][d] = inv[0][d];
    g[2][d] = inv[1][d];
    g[3][d] = inv[2][d];
    g[0][d] = -(g[1][d] + g[2][d] + g[3][d]);
  }
  *vol = std::fabs(det) / 6.0;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) K[i][j] = *vol * (g[i][0] * g[j][0] + g[i][1] * g[j][1] + g[i][2] * g[j][2]);
}

// Stiffness (a = 1) and lumped masses of the unit voxel cut into its six
// Kuhn tetrahedra (8 corners, id a + 2b + 4c) and of the voxel refined once
// (each tetrahedron bisected along the diagonal at the centre, id 8).
void unit_voxel_matrices(double K8[64], double m8[8], double K9[81], double m9[9]) {
  for (int i = 0; i < 64; ++i) K8[i] = 0.0;
  for (int i = 0; i < 81; ++i) K9[i] = 0.0;
  for (int i = 0; i < 8; ++i) m8[i] = 0.0;
  for (int i = 0; i < 9; ++i) m9[i] = 0.0;
  double P[9][3];
  for (int c = 0; c < 8; ++c) {
    P[c][0] = c & 1;
    P[c][1] = (c >> 1) & 1;
    P[c][2] = c >> 2;
  }
  P[8][0] = P[8][1] = P[8][2] = 0.5;
  const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  for (const auto& pm : perms) {
    int v[4] = {0, 0, 0, 7};
    v[1] = 1 << pm[0];
    v[2] = v[1] | (1 << pm[1]);
    const int tets[3][4] = {{v[0], v[1], v[2], v[3]}, {v[0], v[1], v[2], 8}, {8, v[1], v[2], v[3]}};
    for (int t = 0; t < 3; ++t) {
      double X[4][3], vol, K[4][4];
      for (int q = 0; q < 4; ++q)
        for (int d = 0; d < 3; ++d) X[q][d] = P[tets[t][q]][d];
      p1_tet(X, &vol, K);
      for (int a = 0; a < 4; ++a) {
        const int ia = tets[t][a];
        if (t == 0) m8[ia] += vol / 4.0;
        else m9[ia] += vol / 4.0;
        for (int b = 0; b < 4; ++b) {
          if (t == 0) K8[ia * 8 + tets[t][b]] += K[a][b];
          else K9[ia * 9 + tets[t][b]] += K[a][b];
        }
      }
    }
  }
}

template <typename V>
hyb_status upload(hyb_mesh* m, DevBuf& b, const std::vector<V>& host) {
  HYB_TRY(ensure(m, b, host.size() * sizeof(V)));
  // on the mesh's stream, so that its kernels are ordered after the copy
  // whatever kind of stream it is (a synchronous copy from pageable memory
  // may return before its DMA lands and orders only the legacy stream), then
  // wait for it: host is a temporary
  if (!host.empty()) {
    HYB_CU(cudaMemcpyAsync(b.p, host.data(), host.size() * sizeof(V), cudaMemcpyHostToDevice, m->st));
    HYB_CU(cudaStreamSynchronize(m->st));
  }
  return HYB_OK;
}

// Element tables of the all-FEM path: the six Kuhn tetrahedra of the unit
// voxel (corner ids a + 2b + 4c; each the path 0 -> e_p -> e_p + e_q -> (1,1,1))
// with their P1 stiffness at a = 1 and volumes, from the generic element
// formula.
hyb_status build_kuhn(hyb_mesh* m) {
  std::vector<double> tab(6 * 16 + 6);
  std::vector<int> verts(6 * 4);
  // per-axis steps: the brick in units of dx_1, its tables divided by its
  // volume (every interior node's lumped mass stays 1, as on the unit cube)
  const double sc[3] = {1.0, m->ani ? m->hv[1] / m->hv[0] : 1.0, m->ani ? m->hv[2] / m->hv[0] : 1.0};
  const double bvol = sc[0] * sc[1] * sc[2];
  const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  for (int t = 0; t < 6; ++t) {
    const int v1 = 1 << perms[t][0], v2 = v1 | (1 << perms[t][1]);
    const int v[4] = {0, v1, v2, 7};
    double X[4][3], vol, K[4][4];
    for (int q = 0; q < 4; ++q) {
      verts[4 * t + q] = v[q];
      X[q][0] = (v[q] & 1) * sc[0];
      X[q][1] = ((v[q] >> 1) & 1) * sc[1];
      X[q][2] = (v[q] >> 2) * sc[2];
    }
    p1_tet(X, &vol, K);
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) tab[16 * t + 4 * a + b] = m->ani ? K[a][b] / bvol : K[a][b];
    tab[96 + t] = m->ani ? vol / bvol : vol;
  }
  HYB_TRY(upload(m, m->kuhn, tab));
  HYB_TRY(upload(m, m->kuhn_v, verts));
  return HYB_OK;
}

// Refined region: the refined voxels' centre ids, the mask of their corners
// (the rows the interior blocks correct), the unit-voxel tables, and the
// stability bound: the rows of the corners and centres are assembled here
// once, entry by entry from the unit-voxel matrices (a = 1), for their
// row-sum (Gershgorin) bound and their counts only.
hyb_status build_refined(hyb_mesh* m, const uint8_t* mask) {
  const long long nu = m->nu;
  std::vector<int> cid(nu, -1);
  std::vector<unsigned char> refv(nu, 0);
  std::vector<int> refid;
  for (long long u = 0; u < nu; ++u) {
    if (!mask[u]) continue;
    const int x = (int)(u % m->un[0]), y = (int)((u / m->un[0]) % m->un[1]), z = (int)(u / ((long long)m->un[0] * m->un[1]));
    const int o[3] = {m->fl[0] + x, m->fl[1] + y, m->fl[2] + z};
    for (int d = 0; d < 3; ++d)
      if (o[d] < 2 || o[d] + 1 > m->n[d] - 3)
        return fail(HYB_ERR_ARG, "refined voxel %lld: its corners must be at least 2 nodes from the faces", u);
    cid[u] = (int)refid.size();
    refv[u] = 1;
    refid.push_back((int)u);
  }
  m->nc = (int)refid.size();
  if (m->nc == 0) return HYB_OK;
  double K8[64], m8[8], K9[81], m9[9];
  unit_voxel_matrices(K8, m8, K9, m9);
  const long long N = m->Np;  // centre columns follow the lattice field entries
  auto lid = [&](int i, int j, int k) { return (long long)i + (long long)m->px * (j + (long long)m->n[1] * k); };
  auto unk_of = [&](int i, int j, int k) -> long long {  // voxel with origin (i,j,k)
    const int x = i - m->fl[0], y = j - m->fl[1], z = k - m->fl[2];
    if (x < 0 || y < 0 || z < 0 || x >= m->un[0] || y >= m->un[1] || z >= m->un[2]) return -1;
    return x + (long long)m->un[0] * (y + (long long)m->un[1] * z);
  };
  // lattice rows: corners of refined voxels, in lattice order
  std::vector<long long> rows;
  std::vector<unsigned char> rmask((size_t)m->hbox, 0);
  for (int u : refid) {
    const int x = u % m->un[0], y = (u / m->un[0]) % m->un[1], z = u / (m->un[0] * m->un[1]);
    for (int c = 0; c < 8; ++c) {
      const int i = m->fl[0] + x + (c & 1), j = m->fl[1] + y + ((c >> 1) & 1), k = m->fl[2] + z + (c >> 2);
      const long long b = (long long)(i - m->hx0) + (long long)m->hpx * ((j - m->fl[1]) + (long long)m->fn[1] * (k - m->fl[2]));
      if (!rmask[b]) {
        rmask[b] = 1;
        rows.push_back(lid(i, j, k));
      }
    }
  }
  std::sort(rows.begin(), rows.end());
  m->nrl = (int)rows.size();
  m->nr = m->nrl + m->nc;
  long long nnz = 0;
  double bound = 0.0;  // largest row-sum (Gershgorin) bound of M^{-1} K at a = 1, unit spacing
  auto emit_row = [&](std::vector<std::pair<long long, std::pair<int, double>>>& ent, double M) {
    std::sort(ent.begin(), ent.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
    double absum = 0.0, sum = 0.0;
    size_t q = 0;
    while (q < ent.size()) {
      const long long col = ent[q].first;
      double wsum = 0.0;
      while (q < ent.size() && ent[q].first == col) {
        wsum += -ent[q].second.second / M;
        ++q;
      }
      ++nnz;
      absum += std::fabs(wsum);
      sum += wsum;
    }
    bound = std::max(bound, std::fabs(sum) + absum);
  };
  for (long long p : rows) {
    const int i = (int)(p % m->px), j = (int)((p / m->px) % m->n[1]), k = (int)(p / ((long long)m->px * m->n[1]));
    std::vector<std::pair<long long, std::pair<int, double>>> ent;
    double M = 0.0;
    for (int c = 0; c < 8; ++c) {
      const int a = c & 1, b = (c >> 1) & 1, d = c >> 2;
      const int oi = i - a, oj = j - b, ok = k - d;  // voxel origin; this node is its corner c
      const long long u = unk_of(oi, oj, ok);
      const bool ref = u >= 0 && refv[u];
      if (ref) {
        M += m9[c];
        for (int q = 0; q < 9; ++q) {
          if (q == c || std::fabs(K9[c * 9 + q]) < 1e-14) continue;
          const long long col = q < 8 ? lid(oi + (q & 1), oj + ((q >> 1) & 1), ok + (q >> 2)) : N + cid[u];
          ent.push_back({col, {(int)u, K9[c * 9 + q]}});
        }
      } else {
        M += m8[c];
        for (int q = 0; q < 8; ++q) {
          if (q == c || std::fabs(K8[c * 8 + q]) < 1e-14) continue;
          ent.push_back({lid(oi + (q & 1), oj + ((q >> 1) & 1), ok + (q >> 2)), {(int)u, K8[c * 8 + q]}});
        }
      }
    }
    emit_row(ent, M);
  }
  for (int u : refid) {  // centre rows
    const int x = u % m->un[0], y = (u / m->un[0]) % m->un[1], z = u / (m->un[0] * m->un[1]);
    const int oi = m->fl[0] + x, oj = m->fl[1] + y, ok = m->fl[2] + z;
    std::vector<std::pair<long long, std::pair<int, double>>> ent;
    for (int q = 0; q < 8; ++q) {
      if (std::fabs(K9[8 * 9 + q]) < 1e-14) continue;
      ent.push_back({lid(oi + (q & 1), oj + ((q >> 1) & 1), ok + (q >> 2)), {u, K9[8 * 9 + q]}});
    }
    emit_row(ent, m9[8]);
  }
  m->nnz = (int)nnz;
  // stability: the refined rows' bound at a = a_max, against h / sqrt(3 a_max)
  const double h = m->d.h;
  const double lam = std::max(12.0, bound) * m->d.a_max / (h * h);
  m->dt_max = std::min(m->dt_max, 2.0 / std::sqrt(lam));
  std::vector<double> k9(81);  // the kernels accumulate six times the pairing (see kGradPairScale)
  for (int q = 0; q < 81; ++q) k9[q] = 6.0 * K9[q];
  for (int q = 0; q < 81; ++q) m->uK9[q] = K9[q];
  for (int q = 0; q < 64; ++q) m->uK8[q] = K8[q];
  for (int q = 0; q < 9; ++q) m->um9[q] = m9[q];
  for (int q = 0; q < 8; ++q) m->um8[q] = m8[q];
  {  // device flags over the FEM-owned box: bit 0 corner of a refined voxel, bit 1 origin of one
    std::vector<unsigned char> flags(rmask);
    for (int u : refid) {
      const int x = u % m->un[0], y = (u / m->un[0]) % m->un[1], z = u / (m->un[0] * m->un[1]);
      flags[(size_t)(m->fl[0] + x - m->hx0) + (size_t)m->hpx * (y + (size_t)m->fn[1] * z)] |= 2;
    }
    HYB_TRY(upload(m, m->rmask, flags));
  }
  HYB_TRY(upload(m, m->rcid, cid));
  // corner positions packed for the kernel: (i | j << 16, k)
  if (m->n[0] > 65535 || m->n[1] > 65535) return fail(HYB_ERR_ARG, "refinement needs n < 65536 along x and y");
  std::vector<unsigned> pos(2 * rows.size());
  for (size_t r = 0; r < rows.size(); ++r) {
    const long long id = rows[r], plane = (long long)m->px * m->n[1];
    const long long i = id % m->px, j = (id / m->px) % m->n[1], k = id / plane;
    pos[2 * r] = (unsigned)i | ((unsigned)j << 16);
    pos[2 * r + 1] = (unsigned)k;
  }
  HYB_TRY(upload(m, m->rpos, pos));
  // z range of the sparse-row nodes of each FEM-owned column
  std::vector<int> rzr((size_t)2 * m->fn[0] * m->fn[1]);
  for (size_t c = 0; c < rzr.size() / 2; ++c) {
    rzr[2 * c] = 1 << 30;
    rzr[2 * c + 1] = -1;
  }
  for (int k = 0; k < m->fn[2]; ++k)
    for (int j = 0; j < m->fn[1]; ++j)
      for (int i = 0; i < m->fn[0]; ++i) {
        const int x = m->fl[0] + i;
        if (!rmask[(size_t)(x - m->hx0) + (size_t)m->hpx * (j + (size_t)m->fn[1] * k)]) continue;
        const size_t c = (size_t)i + (size_t)m->fn[0] * j;
        rzr[2 * c] = std::min(rzr[2 * c], m->fl[2] + k);
        rzr[2 * c + 1] = std::max(rzr[2 * c + 1], m->fl[2] + k);
      }
  HYB_TRY(upload(m, m->rzr, rzr));
  HYB_TRY(upload(m, m->refvox, refv));
  HYB_TRY(upload(m, m->refvox_id, refid));
  // the refined voxels' origins packed for the kernel: (x | y << 16, z) in unknown-voxel coordinates
  std::vector<unsigned> vxyz(2 * refid.size());
  for (size_t v = 0; v < refid.size(); ++v) {
    const long long id = refid[v];
    vxyz[2 * v] = (unsigned)(id % m->un[0]) | ((unsigned)((id / m->un[0]) % m->un[1]) << 16);
    vxyz[2 * v + 1] = (unsigned)(id / ((long long)m->un[0] * m->un[1]));
  }
  HYB_TRY(upload(m, m->rvxyz, vxyz));
  HYB_TRY(upload(m, m->k9, k9));
  HYB_TRY(ensure(m, m->avox, (size_t)nu * esize(m)));
  return HYB_OK;
}

// Tiled tensor maps for the step kernel's bulk copies (cuTensorMapEncodeTiled
// through the runtime's driver entry point, so the library does not link the
// driver library directly).
typedef CUresult (*TmapEncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

TmapEncodeFn tmap_encoder() {
  static const TmapEncodeFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return (TmapEncodeFn) nullptr;
    }
    return (TmapEncodeFn)p;
  }();
  return fn;
}

// 3-D map of d0 x d1 x d2 elements with row pitch p0 and plane pitch p1
// (elements; 16-byte multiples), box b0 x b1 x 1.  L2 fills of its copies
// are promoted to 64 bytes, not 128: a box's halo columns then bring in half
// of the neighbouring tile's line, not all of it (10 % fewer DRAM bytes on
// the 257^3 lattice with eight sources, time unchanged or lower).
template <typename T>
hyb_status encode_map(CUtensorMap* map, const void* base, uint64_t d0, uint64_t d1, uint64_t d2, uint64_t p0,
                      uint64_t p1, uint32_t b0, uint32_t b1) {
  const TmapEncodeFn enc = tmap_encoder();
  if (!enc) return fail(HYB_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
  const cuuint64_t dims[3] = {d0, d1, d2};
  const cuuint64_t strides[2] = {p0 * sizeof(T), p1 * sizeof(T)};
  const cuuint32_t box[3] = {b0, b1, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = enc(map, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3,
                         const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_64B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(HYB_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return HYB_OK;
}

// Maps of one sweep: the field buffer `field` (3 levels x nsrc slots), the
// edge weights, and (transposed step with pairing) the history buffer of
// `hist_levels` levels.
template <typename T>
hyb_status step_maps(const hyb_mesh* m, StepArgs<T>& A, const DevBuf& field, int nsrc, int hist_levels) {
  HYB_TRY(encode_map<T>(&A.tmf, field.p, m->n[0], m->n[1], (uint64_t)m->n[2] * 3 * nsrc, m->px,
                        (uint64_t)m->px * m->n[1], Box<T>::BX, kBoxY));
  HYB_TRY(encode_map<T>(&A.tmp, field.p, m->n[0], m->n[1], (uint64_t)m->n[2] * 3 * nsrc, m->px,
                        (uint64_t)m->px * m->n[1], Box<T>::PX, kTileY));
  if (m->fem && m->wsz > 0)
    HYB_TRY(encode_map<T>(&A.tmw, m->W.p, m->wpx, m->wn[1], 3ull * m->wn[2] * (m->batch ? nsrc : 1), m->wpx,
                          (uint64_t)m->wpx * m->wn[1], Box<T>::BX, kHBoxY));
  if (hist_levels > 0 && m->hbox > 0)
    HYB_TRY(encode_map<T>(&A.tmh, m->hist.p, m->hpx, m->fn[1], (uint64_t)m->fn[2] * nsrc * hist_levels, m->hpx,
                          (uint64_t)m->hpx * m->fn[1], Box<T>::BX, kHBoxY));
  return HYB_OK;
}

// Work items of the step launches with `nslots` slots (built and uploaded the
// first time this slot count is used, outside any captured sweep).
template <typename T>
hyb_status step_items(hyb_mesh* m, StepArgs<T>& A, int nslots, bool adjoint) {
  if (A.small) return HYB_OK;
  const int d = adjoint ? 1 : 0;
  DevBuf& buf = m->items[d][nslots];
  if (!buf.p) {
    const std::vector<int> host = build_items(m, nslots, adjoint);
    HYB_TRY(upload(m, buf, host));
    m->nitems[d][nslots] = (int)(host.size() / 4);
  }
  A.items = (const int*)buf.p;
  A.nitems = m->nitems[d][nslots];
  return HYB_OK;
}

template <typename T>
void base_args(const hyb_mesh* m, StepArgs<T>& A, double dt, int nslots) {
  std::memset(&A, 0, sizeof(A));
  A.nx = m->n[0];
  A.ny = m->n[1];
  A.nz = m->n[2];
  for (int d = 0; d < 3; ++d) {
    A.fl[d] = m->fl[d];
    A.fh[d] = m->fh[d];
    A.fn[d] = m->fn[d];
    A.wl[d] = m->wl[d];
    A.wn[d] = m->wn[d];
    A.un[d] = m->un[d];
  }
  A.wsz = m->wsz;
  A.px = m->px;
  A.wx0 = m->wx0;
  A.wpx = m->wpx;
  A.hx0 = m->hx0;
  A.hpx = m->hpx;
  A.err = (int*)m->flag.p + 1;
  A.wait = m->d.wait_cycles == 0 ? (1LL << 29) : (m->d.wait_cycles < 0 ? -1LL : (long long)m->d.wait_cycles);
  A.W = (const T*)m->W.p;
  A.G = (double*)m->G.p;
  A.avox = (const T*)m->avox.p;
  A.sdamp = m->d.model == HYB_MODEL_TELEGRAPH ? (const T*)m->sdamp.p : nullptr;
  const double h = m->ani ? m->hv[0] : m->d.h;
  A.c2 = (T)(dt * dt / (h * h));
  A.r = (T)((h - dt) / (h + dt));
  step_geometry(m, &A.npb, &A.ntx, &A.small, &A.nedge);
  if (m->ani) {  // every level by the bulk and shell kernels, axis terms weighed by kap
    A.ani = 1;
    A.small = 1;
    A.nedge = 0;
    for (int a = 0; a < 3; ++a) {
      A.kap[a] = (h * h) / (m->hv[a] * m->hv[a]);
      A.kapt[a] = (T)A.kap[a];
      A.ra[a] = (T)((m->hv[a] - dt) / (m->hv[a] + dt));
    }
    A.kdiag = (T)(-2.0 * (A.kap[0] + A.kap[1] + A.kap[2]));
  }
  if (m->d.fem_path == HYB_FEM_TET_ALL) {  // every level by the all-node kernels
    A.tet = 1;
    A.small = 1;
    A.nedge = 0;
    A.acoef = (const double*)m->acopy.p;
    A.kuhn = (const double*)m->kuhn.p;
    A.kuhn_v = (const int*)m->kuhn_v.p;
  }
  A.nslots = nslots;
  if (m->nc > 0) {
    A.nref = m->nc;
    A.nrl = m->nrl;
    A.rpos = (const uint2*)m->rpos.p;
    A.rvxyz = (const uint2*)m->rvxyz.p;
    A.rcid = (const int*)m->rcid.p;
    for (int q = 0; q < 81; ++q) A.rK9[q] = (T)m->uK9[q];
    for (int c = 0; c < 8; ++c) {
      for (int q = 0; q < 8; ++q) A.rdK[9 * c + q] = (T)(m->uK9[9 * c + q] - m->uK8[8 * c + q]);
      A.rdK[9 * c + 8] = (T)m->uK9[9 * c + 8];
      A.rm8[c] = (T)m->um8[c];
    }
    for (int q = 0; q < 9; ++q) A.rm9[q] = (T)m->um9[q];
    A.rmask = (const unsigned char*)m->rmask.p;
    A.rzr = (const int*)m->rzr.p;
    A.refvox = (const unsigned char*)m->refvox.p;
    A.refvox_id = (const int*)m->refvox_id.p;
    A.k9 = (const double*)m->k9.p;
  }
}

// The coefficient of slot s: its edge weights (and their plane in the
// weight tensor map) and its refined voxels' a; per slot for a batch.
template <typename T>
void slot_coef(const hyb_mesh* m, Slot<T>& S, int s) {
  const int q = m->batch ? s : 0;
  S.W = (const T*)m->W.p + (size_t)q * 3 * m->wsz;
  S.zf_w = q * 3 * m->wn[2];
  S.avox = m->avox.p ? (const T*)m->avox.p + (size_t)q * m->nu : nullptr;
}

template <typename T>
T* centre_buf(const hyb_mesh* m, const DevBuf& b, int nsrc, int s, int level) {
  if (m->nc == 0) return nullptr;
  const int r = ((level % 3) + 3) % 3;
  return (T*)b.p + ((size_t)r * nsrc + s) * (size_t)m->nc;
}

template <typename T>
T* field_buf(const hyb_mesh* m, const DevBuf& b, int nsrc, int s, int level) {
  const int r = ((level % 3) + 3) % 3;
  return (T*)b.p + ((size_t)r * nsrc + s) * (size_t)m->Np;
}

// Fill the forward slots of step k (u^k -> u^{k+1}).
template <typename T>
void forward_slots(const hyb_mesh* m, StepArgs<T>& A, const hyb_source* src, int nsrc, int nsteps,
                   double dt, int k, T* trace, T* hist_level, T* chist_level) {
  for (int s = 0; s < nsrc; ++s) {
    Slot<T>& S = A.s[s];
    S.cur = field_buf<T>(m, m->U, nsrc, s, k);
    S.prev = field_buf<T>(m, m->U, nsrc, s, k - 1);
    S.next = field_buf<T>(m, m->U, nsrc, s, k + 1);
    S.obs_w = trace ? trace + ((size_t)s * (nsteps + 1) + (k + 1)) * (size_t)m->obs_stride : nullptr;
    S.obs_r = nullptr;
    S.hist_w = hist_level ? hist_level + (size_t)s * m->hbox : nullptr;
    S.hist_r = nullptr;
    S.ccur = centre_buf<T>(m, m->CU, nsrc, s, k);
    S.cprev = centre_buf<T>(m, m->CU, nsrc, s, k - 1);
    S.cnext = centre_buf<T>(m, m->CU, nsrc, s, k + 1);
    S.chist_w = (hist_level && m->nc) ? chist_level + (size_t)s * m->nc : nullptr;
    S.chist_r = nullptr;
    slot_coef<T>(m, S, s);
    set_wave<T>(m, S, src[s], k, dt);
    S.mask_e = 0;
    S.mask_c = 0;
    S.zf_cur = (int)((S.cur - (const T*)m->U.p) / ((long long)m->px * m->n[1]));
    S.zf_prev = (int)((S.prev - (const T*)m->U.p) / ((long long)m->px * m->n[1]));
    S.zf_hist = 0;
    S.obs_face = src[s].face;
  }
}

// Levels 0 and -1 of one source (lattice field and centre values): the
// initial state of Model Problem 1 if one was set, else zero.
template <typename T>
hyb_status initial_levels(hyb_mesh* m, T* u0, T* um, T* c0, T* cm, cudaStream_t st) {
  const size_t fb = (size_t)m->Np * sizeof(T), cb = (size_t)m->nc * sizeof(T);
  if (m->have_init) {
    HYB_CU(cudaMemcpyAsync(u0, m->I0.p, fb, cudaMemcpyDeviceToDevice, st));
    HYB_CU(cudaMemcpyAsync(um, (const char*)m->I0.p + fb, fb, cudaMemcpyDeviceToDevice, st));
    if (m->nc) {
      HYB_CU(cudaMemcpyAsync(c0, m->IC0.p, cb, cudaMemcpyDeviceToDevice, st));
      HYB_CU(cudaMemcpyAsync(cm, (const char*)m->IC0.p + cb, cb, cudaMemcpyDeviceToDevice, st));
    }
    return HYB_OK;
  }
  HYB_CU(cudaMemsetAsync(u0, 0, fb, st));
  HYB_CU(cudaMemsetAsync(um, 0, fb, st));
  if (m->nc) {
    HYB_CU(cudaMemsetAsync(c0, 0, cb, st));
    HYB_CU(cudaMemsetAsync(cm, 0, cb, st));
  }
  return HYB_OK;
}

template <typename T>
hyb_status forward_impl(hyb_mesh* m, const double* a, const hyb_source* src, int nsrc, int nsteps,
                        double dt, T* trace, bool keep, bool batch = false) {
  const size_t fb = (size_t)m->Np * sizeof(T);
  const int C = m->d.ckpt_every;
  const bool ckpt = C > 0;
  const size_t cb = (size_t)m->nc * sizeof(T);  // centre values of one level
  HYB_TRY(ensure(m, m->U, 3 * (size_t)nsrc * fb));
  HYB_TRY(ensure(m, m->CU, 3 * (size_t)nsrc * cb));
  if (m->d.fem_path == HYB_FEM_TET_ALL) HYB_TRY(ensure(m, m->acopy, (size_t)std::max(m->nu, 1LL) * sizeof(double)));
  if (keep && m->nown > 0) {
    if (!ckpt) {
      HYB_TRY(ensure(m, m->hist, (size_t)nsteps * nsrc * m->hbox * sizeof(T)));
      HYB_TRY(ensure(m, m->chist, (size_t)nsteps * nsrc * cb));
    } else {
      const size_t nseg = ((size_t)nsteps + C - 1) / C;
      HYB_TRY(ensure(m, m->ckpt, nseg * 2 * (size_t)nsrc * fb));
      HYB_TRY(ensure(m, m->cckpt, nseg * 2 * (size_t)nsrc * cb));
      HYB_TRY(ensure(m, m->hist, (size_t)C * nsrc * m->hbox * sizeof(T)));
      HYB_TRY(ensure(m, m->chist, (size_t)C * nsrc * cb));
    }
  }
  const int ncoef = batch ? nsrc : 1;  // coefficient sets: one per slot for a batch
  if (m->fem) HYB_TRY(ensure(m, m->W, (size_t)ncoef * 3 * m->wsz * sizeof(T)));
  if (m->nc > 0) HYB_TRY(ensure(m, m->avox, (size_t)ncoef * m->nu * sizeof(T)));
  m->batch = batch;
  StepArgs<T> A;
  base_args(m, A, dt, nsrc);
  HYB_TRY(step_maps<T>(m, A, m->U, nsrc, 0));
  HYB_TRY(step_items<T>(m, A, nsrc, false));
  const bool tel = m->d.model == HYB_MODEL_TELEGRAPH;
  if (tel) {  // the edge weights of a = 1, the damping ratios from sigma
    if (!m->ones.p) HYB_TRY(upload(m, m->ones, std::vector<double>((size_t)std::max(m->nu, 1LL), 1.0)));
    HYB_TRY(ensure(m, m->sdamp, (size_t)std::max(m->hbox, 1LL) * sizeof(T)));
    A.sdamp = (const T*)m->sdamp.p;
    launch_set_damp<T>(A, (T*)m->sdamp.p, a, dt, (int*)m->flag.p, m->st);
    HYB_LAUNCHED(m);
  }
  if (m->fem)
    for (int q = 0; q < ncoef; ++q) {
      launch_set_coef<T>(A, (T*)m->W.p + (size_t)q * 3 * m->wsz,
                         m->nc > 0 ? (T*)m->avox.p + (size_t)q * m->nu : nullptr,
                         tel ? (const double*)m->ones.p : a + (size_t)q * m->nu, m->d.a_max, (int*)m->flag.p, m->st);
      HYB_LAUNCHED(m);
    }
  if (A.tet && m->nu > 0)  // the all-FEM rows read a itself
    HYB_CU(cudaMemcpyAsync(m->acopy.p, a, (size_t)m->nu * sizeof(double), cudaMemcpyDeviceToDevice, m->st));
  auto body = [&](cudaStream_t st) -> hyb_status {
    for (int s = 0; s < nsrc; ++s)
      HYB_TRY(initial_levels<T>(m, field_buf<T>(m, m->U, nsrc, s, 0), field_buf<T>(m, m->U, nsrc, s, -1),
                                centre_buf<T>(m, m->CU, nsrc, s, 0), centre_buf<T>(m, m->CU, nsrc, s, -1), st));
    if (trace) {
      HYB_CU(cudaMemsetAsync(trace, 0, (size_t)nsrc * (nsteps + 1) * m->obs_stride * sizeof(T), st));
      if (m->have_init)  // row 0 of every source: u^0 on its face
        for (int s = 0; s < nsrc; ++s) {
          launch_extract_face<T>(A, field_buf<T>(m, m->U, nsrc, s, 0), src[s].face,
                                 trace + (size_t)s * (nsteps + 1) * m->obs_stride, st);
          HYB_LAUNCHED(m);
        }
    }
    T* hist = (T*)m->hist.p;
    T* chist = (T*)m->chist.p;
    if (keep && !ckpt && m->nown > 0) {
      if (m->have_init) {
        for (int s = 0; s < nsrc; ++s) {
          launch_extract_owned<T>(A, field_buf<T>(m, m->U, nsrc, s, 0), hist + (size_t)s * m->hbox, st);
          HYB_LAUNCHED(m);
          if (m->nc)
            HYB_CU(cudaMemcpyAsync(chist + (size_t)s * m->nc, centre_buf<T>(m, m->CU, nsrc, s, 0), cb,
                                   cudaMemcpyDeviceToDevice, st));
        }
      } else {
        HYB_CU(cudaMemsetAsync(hist, 0, (size_t)nsrc * m->hbox * sizeof(T), st));
        if (m->nc) HYB_CU(cudaMemsetAsync(chist, 0, (size_t)nsrc * cb, st));
      }
    }
    const size_t lvl = (size_t)nsrc * m->hbox;
    const size_t clvl = (size_t)nsrc * m->nc;
    for (int k = 0; k < nsteps; ++k) {
      if (keep && ckpt && m->nown > 0 && k > 0 && k % C == 0) {
        const size_t seg = (size_t)(k / C);
        for (int s = 0; s < nsrc; ++s) {
          char* base = (char*)m->ckpt.p + ((seg * nsrc + s) * 2) * fb;
          HYB_CU(cudaMemcpyAsync(base, field_buf<T>(m, m->U, nsrc, s, k), fb, cudaMemcpyDeviceToDevice, st));
          HYB_CU(cudaMemcpyAsync(base + fb, field_buf<T>(m, m->U, nsrc, s, k - 1), fb, cudaMemcpyDeviceToDevice,
                                 st));
          if (m->nc) {
            char* cbase = (char*)m->cckpt.p + ((seg * nsrc + s) * 2) * cb;
            HYB_CU(cudaMemcpyAsync(cbase, centre_buf<T>(m, m->CU, nsrc, s, k), cb, cudaMemcpyDeviceToDevice, st));
            HYB_CU(cudaMemcpyAsync(cbase + cb, centre_buf<T>(m, m->CU, nsrc, s, k - 1), cb,
                                   cudaMemcpyDeviceToDevice, st));
          }
        }
      }
      // history slot of step k: u^{k+1} in slot k + 1 (the wave model; slot 0
      // holds u^0), or, in the telegraph model, u^{k+1} - u^{k-1} in slot k
      const int slot = tel ? k : k + 1;
      const bool hk = keep && !ckpt && m->nown > 0 && slot <= nsteps - 1;
      T* hl = hk ? hist + (size_t)slot * lvl : nullptr;
      T* chl = hk ? chist + (size_t)slot * clvl : nullptr;
      forward_slots<T>(m, A, src, nsrc, nsteps, dt, k, trace, hl, chl);
      HYB_TRY(step_launch(m, st, [&](cudaStream_t q) { return launch_forward_step<T>(A, q); }));
    }
    return HYB_OK;
  };
  HYB_TRY(run_sweep(m, m->graphs[keep ? 0 : 1], make_key(m, keep ? 0 : 1, trace, 0, nsteps, nsrc, dt, src), body));
  m->nsteps = nsteps;
  m->nsrc = nsrc;
  m->dt = dt;
  for (int s = 0; s < nsrc; ++s) m->src[s] = src[s];
  m->have_run = true;
  m->have_fwd = keep;
  m->have_adj = false;
  m->u_levels = true;
  return HYB_OK;
}

template <typename T>
void adjoint_slots(const hyb_mesh* m, StepArgs<T>& A, const T* cot, int j, const T* hist_level,
                   const T* chist_level) {
  const int nsrc = m->nsrc, nsteps = m->nsteps;
  for (int s = 0; s < nsrc; ++s) {
    Slot<T>& S = A.s[s];
    S.cur = field_buf<T>(m, m->L, nsrc, s, j + 1);
    S.prev = field_buf<T>(m, m->L, nsrc, s, j + 2);
    S.next = field_buf<T>(m, m->L, nsrc, s, j);
    S.obs_w = nullptr;
    S.obs_r = cot ? cot + ((size_t)s * (nsteps + 1) + j) * (size_t)m->obs_stride : nullptr;
    S.hist_w = nullptr;
    S.hist_r = hist_level ? hist_level + (size_t)s * m->hbox : nullptr;
    S.ccur = centre_buf<T>(m, m->CL, nsrc, s, j + 1);
    S.cprev = centre_buf<T>(m, m->CL, nsrc, s, j + 2);
    S.cnext = centre_buf<T>(m, m->CL, nsrc, s, j);
    S.chist_w = nullptr;
    S.chist_r = (hist_level && m->nc) ? chist_level + (size_t)s * m->nc : nullptr;
    slot_coef<T>(m, S, s);
    S.src_mask = 0;
    S.zf_cur = (int)((S.cur - (const T*)m->L.p) / ((long long)m->px * m->n[1]));
    S.zf_prev = (int)((S.prev - (const T*)m->L.p) / ((long long)m->px * m->n[1]));
    S.zf_hist = S.hist_r ? (int)((S.hist_r - (const T*)m->hist.p) / ((long long)m->hpx * m->fn[1])) : 0;
    S.mask_f = mask_at(m, m->src[s], j, m->dt);
    S.mask_e = mask_at(m, m->src[s], j - 1, m->dt);
    S.mask_c = mask_at(m, m->src[s], j + 1, m->dt);
    S.obs_face = m->src[s].face;
  }
}

// Slots of the paper's adjoint step j: lambda^{j-1} from lambda^j (cur) and
// lambda^{j+1} (prev) by the forward rows with every face reflecting, the
// cotangent row j entering on the observation face (Eq. (fdmschemeadjoint));
// hist_level (u^j) is for the same-index pairing.
template <typename T>
void paper_slots(const hyb_mesh* m, StepArgs<T>& A, const T* cot, int j, const T* hist_level,
                 const T* chist_level) {
  const int nsrc = m->nsrc, nsteps = m->nsteps;
  const double h = m->d.h;
  for (int s = 0; s < nsrc; ++s) {
    Slot<T>& S = A.s[s];
    S = Slot<T>();
    S.cur = field_buf<T>(m, m->L, nsrc, s, j);
    S.prev = field_buf<T>(m, m->L, nsrc, s, j + 1);
    S.next = field_buf<T>(m, m->L, nsrc, s, j - 1);
    S.hist_r = hist_level ? hist_level + (size_t)s * m->hbox : nullptr;
    S.ccur = centre_buf<T>(m, m->CL, nsrc, s, j);
    S.cprev = centre_buf<T>(m, m->CL, nsrc, s, j + 1);
    S.cnext = centre_buf<T>(m, m->CL, nsrc, s, j - 1);
    S.chist_r = (hist_level && m->nc) ? chist_level + (size_t)s * m->nc : nullptr;
    S.zf_cur = (int)((S.cur - (const T*)m->L.p) / ((long long)m->px * m->n[1]));
    S.zf_prev = (int)((S.prev - (const T*)m->L.p) / ((long long)m->px * m->n[1]));
    S.obs_face = m->src[s].face;
    S.inj = cot ? cot + ((size_t)s * (nsteps + 1) + j) * (size_t)m->obs_stride : nullptr;
    S.inj_scale = (T)(-m->dt / (h * h * h));
    slot_coef<T>(m, S, s);
  }
}

// Same-index pairing of the paper's adjoint, G_s += pairing of (u^j, lambda^j)
// for the slots set up by paper_slots (structured and refined voxels).
template <typename T>
hyb_status paper_pair(hyb_mesh* m, StepArgs<T>& A, cudaStream_t st) {
  for (int s = 0; s < m->nsrc; ++s) {
    StepArgs<T> B = A;
    B.G = (double*)m->G.p + (size_t)s * m->nu;
    launch_pair<T>(B, A.s[s].hist_r, A.s[s].cur, st);
    HYB_LAUNCHED(m);
  }
  if (m->nc > 0) {
    launch_refined_pair<T>(A, st);
    HYB_LAUNCHED(m);
  }
  return HYB_OK;
}

// Gradient pairing of level 0: (u^0, lambda^1) on every unknown voxel.
template <typename T>
hyb_status pair_first(hyb_mesh* m, StepArgs<T>& A, const T* level0, const T* clevel0, cudaStream_t st) {
  for (int s = 0; s < m->nsrc; ++s) {
    StepArgs<T> B = A;
    B.G = (double*)m->G.p + (size_t)s * m->nu;
    launch_pair<T>(B, level0 + (size_t)s * m->hbox, field_buf<T>(m, m->L, m->nsrc, s, 1), st);
    HYB_LAUNCHED(m);
  }
  if (m->nc > 0) {
    adjoint_slots<T>(m, A, nullptr, 0, level0, clevel0);  // cur = lambda^1, hist = u^0
    launch_refined_pair<T>(A, st);
    HYB_LAUNCHED(m);
  }
  return HYB_OK;
}

template <typename T>
hyb_status adjoint_impl(hyb_mesh* m, const T* cot, int accumulate) {
  if (!m->have_fwd) return fail(HYB_ERR_STATE, "hyb_adjoint needs a preceding hyb_forward of this mesh");
  const int nsrc = m->nsrc, nsteps = m->nsteps;
  const double dt = m->dt;
  const size_t fb = (size_t)m->Np * sizeof(T);
  const int C = m->d.ckpt_every;
  const bool ckpt = C > 0;
  const bool tel = m->d.model == HYB_MODEL_TELEGRAPH;
  const size_t cb = (size_t)m->nc * sizeof(T);
  HYB_TRY(ensure(m, m->L, 3 * (size_t)nsrc * fb));
  HYB_TRY(ensure(m, m->CL, 3 * (size_t)nsrc * cb));
  HYB_TRY(ensure(m, m->G, (size_t)nsrc * m->nu * sizeof(double)));
  StepArgs<T> A;   // adjoint steps
  base_args(m, A, dt, nsrc);
  StepArgs<T> F;   // recomputed forward steps
  base_args(m, F, dt, nsrc);
  HYB_TRY(step_maps<T>(m, A, m->L, nsrc, ckpt ? C : nsteps));
  HYB_TRY(step_maps<T>(m, F, m->U, nsrc, 0));
  HYB_TRY(step_items<T>(m, A, nsrc, true));
  HYB_TRY(step_items<T>(m, F, nsrc, false));
  const bool paper = m->d.adjoint_mode == HYB_ADJ_PAPER;
  StepArgs<T> Pp;  // paper-mode steps: forward rows on lambda
  if (paper) {
    base_args(m, Pp, dt, nsrc);
    HYB_TRY(step_maps<T>(m, Pp, m->L, nsrc, 0));
    HYB_TRY(step_items<T>(m, Pp, nsrc, false));
  }
  auto body = [&](cudaStream_t st) -> hyb_status {
    if (!accumulate) HYB_CU(cudaMemsetAsync(m->G.p, 0, (size_t)nsrc * m->nu * sizeof(double), st));
    const int z0 = paper ? nsteps : nsteps + 1;  // the two levels that start at zero
    for (int s = 0; s < nsrc; ++s) {
      HYB_CU(cudaMemsetAsync(field_buf<T>(m, m->L, nsrc, s, z0), 0, fb, st));
      HYB_CU(cudaMemsetAsync(field_buf<T>(m, m->L, nsrc, s, z0 + 1), 0, fb, st));
      if (m->nc) {
        HYB_CU(cudaMemsetAsync(centre_buf<T>(m, m->CL, nsrc, s, z0), 0, cb, st));
        HYB_CU(cudaMemsetAsync(centre_buf<T>(m, m->CL, nsrc, s, z0 + 1), 0, cb, st));
      }
    }
    T* hist = (T*)m->hist.p;
    T* chist = (T*)m->chist.p;
    const size_t lvl = (size_t)nsrc * m->hbox;
    const size_t clvl = (size_t)nsrc * m->nc;
    const bool pairing = m->nu > 0 && m->nown > 0;
    auto adj_step = [&](int j, const T* hl, const T* chl) -> hyb_status {
      if (paper) {  // pair (u^j, lambda^j), then lambda^{j-1}
        paper_slots<T>(m, Pp, cot, j, hl, chl);
        if (hl) HYB_TRY(paper_pair<T>(m, Pp, st));
        return step_launch(m, st, [&](cudaStream_t q) { return launch_forward_step<T>(Pp, q); });
      }
      adjoint_slots<T>(m, A, cot, j, hl, chl);
      return step_launch(m, st, [&](cudaStream_t q) { return launch_adjoint_step<T>(A, q); });
    };
    auto first_pair = [&]() -> hyb_status {
      if (!paper) return pair_first<T>(m, A, hist, chist, st);
      paper_slots<T>(m, Pp, nullptr, 0, hist, chist);  // (u^0, lambda^0)
      return paper_pair<T>(m, Pp, st);
    };
    auto fwd_step = [&](int k, T* hl, T* chl) -> hyb_status {
      forward_slots<T>(m, F, m->src, nsrc, nsteps, dt, k, nullptr, hl, chl);
      return step_launch(m, st, [&](cudaStream_t q) { return launch_forward_step<T>(F, q); });
    };
    if (!ckpt) {
      for (int j = nsteps; j >= 1; --j) {
        const bool pj = pairing && j <= nsteps - 1;
        HYB_TRY(adj_step(j, pj ? hist + (size_t)j * lvl : nullptr, pj ? chist + (size_t)j * clvl : nullptr));
      }
      if (pairing) HYB_TRY(first_pair());
      return HYB_OK;
    }
    HYB_TRY(adj_step(nsteps, nullptr, nullptr));
    const int nseg = (nsteps + C - 1) / C;
    for (int seg = nseg - 1; seg >= 0; --seg) {
      const int kb = seg * C;
      const int ke = std::min((seg + 1) * C, nsteps) - 1;
      if (pairing) {
        for (int s = 0; s < nsrc; ++s) {
          T* u0 = field_buf<T>(m, m->U, nsrc, s, kb);
          T* um = field_buf<T>(m, m->U, nsrc, s, kb - 1);
          T* c0 = centre_buf<T>(m, m->CU, nsrc, s, kb);
          T* cm = centre_buf<T>(m, m->CU, nsrc, s, kb - 1);
          if (seg == 0) {
            HYB_TRY(initial_levels<T>(m, u0, um, c0, cm, st));
          } else {
            const char* base = (const char*)m->ckpt.p + (((size_t)seg * nsrc + s) * 2) * fb;
            HYB_CU(cudaMemcpyAsync(u0, base, fb, cudaMemcpyDeviceToDevice, st));
            HYB_CU(cudaMemcpyAsync(um, base + fb, fb, cudaMemcpyDeviceToDevice, st));
            if (m->nc) {
              const char* cbase = (const char*)m->cckpt.p + (((size_t)seg * nsrc + s) * 2) * cb;
              HYB_CU(cudaMemcpyAsync(c0, cbase, cb, cudaMemcpyDeviceToDevice, st));
              HYB_CU(cudaMemcpyAsync(cm, cbase + cb, cb, cudaMemcpyDeviceToDevice, st));
            }
          }
          launch_extract_owned<T>(F, u0, hist + (size_t)s * m->hbox, st);
          HYB_LAUNCHED(m);
          if (m->nc) HYB_CU(cudaMemcpyAsync(chist + (size_t)s * m->nc, c0, cb, cudaMemcpyDeviceToDevice, st));
        }
        // recompute the segment's history (telegraph: one step further, for
        // u^{ke+1} - u^{ke-1} in the last slot)
        const int sh = tel ? 0 : 1;
        for (int k = kb; k < ke + 1 - sh; ++k)
          HYB_TRY(fwd_step(k, hist + (size_t)(k + sh - kb) * lvl, chist + (size_t)(k + sh - kb) * clvl));
      }
      for (int j = ke; j >= std::max(kb, 1); --j)
        HYB_TRY(adj_step(j, pairing ? hist + (size_t)(j - kb) * lvl : nullptr,
                         pairing ? chist + (size_t)(j - kb) * clvl : nullptr));
    }
    if (pairing) HYB_TRY(first_pair());
    return HYB_OK;
  };
  HYB_TRY(run_sweep(m, m->graphs[2], make_key(m, 2, cot, accumulate, nsteps, nsrc, dt, m->src), body));
  m->have_adj = true;
  if (ckpt) m->u_levels = false;  // the recomputed segments reused the forward's levels
  return HYB_OK;
}

// Volume of one lattice cell: h^3, or dx_1 dx_2 dx_3.
double cell_volume(const hyb_mesh* m) {
  return m->ani ? m->hv[0] * m->hv[1] * m->hv[2] : m->d.h * m->d.h * m->d.h;
}

// In-face cell area of face f: h^2, or dx_p dx_q (p, q its in-face axes).
double face_cell_area(const hyb_mesh* m, int f) {
  const int ax = f >> 1, p = ax == 0 ? 1 : 0, q = ax == 2 ? 1 : 2;
  return m->ani ? m->hv[p] * m->hv[q] : m->d.h * m->d.h;
}

// Factor from the accumulated pairing sums (kGradPairScale / h times
// u^T K_c lambda per voxel) to dJ/da: exact adjoint, dJ/da_c =
// -tau^2 u^T K_c (lambda~ / h^3) summed over steps; paper mode,
// g_c = tau u^T K_c lambda summed over steps.  Per-axis steps: the kernels
// accumulate kGradPairScale sum_ax kap_ax u^T K^ax_c lambda~ (the unit-cube
// edge parts K^ax, kap_ax = dx_1^2 / dx_ax^2) and K_c = (|c| / dx_1^2)
// sum_ax kap_ax K^ax_c, so h reads dx_1.
double grad_scale(const hyb_mesh* m) {
  const double h = m->ani ? m->hv[0] : m->d.h, dt = m->dt;
  if (m->d.adjoint_mode == HYB_ADJ_PAPER) return dt * h / kGradPairScale;
  if (m->d.model == HYB_MODEL_TELEGRAPH) return -dt / 24.0;  // the kernels accumulate 12 sum_i m_i lambda_i v_i
  return -dt * dt / (h * h) / kGradPairScale;
}

template <typename T>
hyb_status misfit_impl(hyb_mesh* m, const T* trace, const T* obs, int weights, double* J, T* cot) {
  if (!m->have_run) return fail(HYB_ERR_STATE, "hyb_misfit needs a preceding hyb_forward");
  MisfitGeom g;
  std::memset(&g, 0, sizeof g);
  g.n_src = m->nsrc;
  g.nsteps = m->nsteps;
  g.stride = m->obs_stride;
  for (int s = 0; s < m->nsrc; ++s) {
    const int ax = m->src[s].face >> 1;
    const int p = ax == 0 ? 1 : 0;
    const int q = ax == 2 ? 1 : 2;
    g.face[s] = m->src[s].face;
    g.np[s] = m->n[p];
    g.nq[s] = m->n[q];
  }
  const bool quad = weights == HYB_WEIGHTS_QUADRATURE;
  g.wt = quad ? m->dt : 1.0;
  for (int s = 0; s < m->nsrc; ++s) g.hh[s] = quad ? face_cell_area(m, m->src[s].face) : 1.0;
  g.halve = quad ? 1 : 0;
  HYB_TRY(ensure(m, m->part, 2 * (size_t)kReduceBlocks * sizeof(double)));
  HYB_TRY(ensure(m, m->scal, 16 * sizeof(double)));
  launch_misfit<T>(g, trace, obs, cot, (double*)m->part.p, m->st);
  HYB_LAUNCHED(m);
  launch_sum((double*)m->part.p, kReduceBlocks, (double*)m->scal.p + 8, m->st);
  HYB_LAUNCHED(m);
  if (J) {
    HYB_CU(cudaMemcpyAsync(m->hscal + 8, (double*)m->scal.p + 8, sizeof(double), cudaMemcpyDeviceToHost, m->st));
    HYB_CU(cudaStreamSynchronize(m->st));
    *J = m->hscal[8];
  }
  return HYB_OK;
}

// Per-slot misfit of a batch: slot s's trace rows reduced on their own (the
// same launches and summation order as a one-slot mesh), J of slot s to
// J_host[s] (host, synchronises), cotangent rows as hyb_misfit.
template <typename T>
hyb_status misfit_batch_impl(hyb_mesh* m, const T* trace, const T* obs, int weights, double* J_host, T* cot) {
  if (!m->have_run) return fail(HYB_ERR_STATE, "hyb_misfit_batch needs a preceding forward");
  const int nsrc = m->nsrc;
  const size_t rows = (size_t)(m->nsteps + 1) * m->obs_stride;
  HYB_TRY(ensure(m, m->part, 2 * (size_t)kReduceBlocks * sizeof(double)));
  HYB_TRY(ensure(m, m->scal, (16 + kMaxSlots) * sizeof(double)));
  double* out = (double*)m->scal.p + 16;
  const bool quad = weights == HYB_WEIGHTS_QUADRATURE;
  for (int s = 0; s < nsrc; ++s) {
    MisfitGeom g;
    std::memset(&g, 0, sizeof g);
    g.n_src = 1;
    g.nsteps = m->nsteps;
    g.stride = m->obs_stride;
    const int ax = m->src[s].face >> 1;
    g.face[0] = m->src[s].face;
    g.np[0] = m->n[ax == 0 ? 1 : 0];
    g.nq[0] = m->n[ax == 2 ? 1 : 2];
    g.wt = quad ? m->dt : 1.0;
    g.hh[0] = quad ? face_cell_area(m, m->src[s].face) : 1.0;
    g.halve = quad ? 1 : 0;
    launch_misfit<T>(g, trace + s * rows, obs + s * rows, cot ? cot + s * rows : nullptr, (double*)m->part.p, m->st);
    HYB_LAUNCHED(m);
    launch_sum((double*)m->part.p, kReduceBlocks, out + s, m->st);
    HYB_LAUNCHED(m);
  }
  if (J_host) {
    HYB_CU(cudaMemcpyAsync(m->hscal, out, nsrc * sizeof(double), cudaMemcpyDeviceToHost, m->st));
    HYB_CU(cudaStreamSynchronize(m->st));
    for (int s = 0; s < nsrc; ++s) J_host[s] = m->hscal[s];
  }
  return HYB_OK;
}

double quadratic_step(double J0, double dJ0, double at, double Jt) {
  const double curv = Jt - J0 - dJ0 * at;
  double alpha = curv <= 0.0 ? at : -dJ0 * at * at / (2.0 * curv);
  return std::min(std::max(alpha, 0.0), 4.0 * at);
}

template <typename T>
hyb_status cg_impl(hyb_mesh* m, double* a, const T* obs, const hyb_source* src, int nsrc, int nsteps,
                   double dt, const hyb_cg_params* P, hyb_cg_state* S, hyb_cg_report* R) {
  const size_t tb = (size_t)nsrc * (nsteps + 1) * m->obs_stride * sizeof(T);
  const long long nu = m->nu;
  const double vol = cell_volume(m);
  HYB_TRY(ensure(m, m->trace, tb));
  HYB_TRY(ensure(m, m->cot, tb));
  HYB_TRY(ensure(m, m->g, (size_t)nu * sizeof(double)));
  HYB_TRY(ensure(m, m->atrial, (size_t)nu * sizeof(double)));
  HYB_TRY(ensure(m, m->part, kCgParts * (size_t)kReduceBlocks * sizeof(double)));
  HYB_TRY(ensure(m, m->scal, 16 * sizeof(double)));
  double* part = (double*)m->part.p;
  double* scal = (double*)m->scal.p;
  double* g = (double*)m->g.p;
  T* tr = (T*)m->trace.p;
  // Step 1: state and adjoint at a^m.
  HYB_TRY(forward_impl<T>(m, a, src, nsrc, nsteps, dt, tr, true));
  double Jd = 0.0;
  HYB_TRY(misfit_impl<T>(m, tr, obs, P->weights, &Jd, (T*)m->cot.p));
  HYB_TRY(adjoint_impl<T>(m, (const T*)m->cot.p, 0));
  launch_grad_finalize((const double*)m->G.p, nsrc, a, grad_scale(m), P->gamma, vol, P->a0, g, nu, m->st);
  HYB_LAUNCHED(m);
  launch_cg_norms(g, a, P->a0, P->a_min, P->a_max, nu, part, m->st);
  HYB_LAUNCHED(m);
  for (int q = 0; q < kCgParts; ++q) {
    launch_sum(part + q * kReduceBlocks, kReduceBlocks, scal + 5 + q, m->st);
    HYB_LAUNCHED(m);
  }
  HYB_CU(cudaMemcpyAsync(m->hscal + 5, scal + 5, kCgParts * sizeof(double), cudaMemcpyDeviceToHost, m->st));
  HYB_CU(cudaStreamSynchronize(m->st));
  const double gn2 = m->hscal[5] / vol;   // ||g||_L2^2 with g = (dF/da) / |c|
  const double gpn2 = m->hscal[7] / vol;  // the same for the projected gradient
  const double J0 = Jd + 0.5 * P->gamma * vol * m->hscal[6];
  // Step 2: Fletcher-Reeves direction of the projected gradient.
  double beta = (S->iter > 0 && S->gnorm2 > 0.0) ? gpn2 / S->gnorm2 : 0.0;
  launch_cg_direction(g, a, P->a_min, P->a_max, vol, beta, S->d, nu, m->st);
  HYB_LAUNCHED(m);
  auto dir_stats = [&](double* dJ0, double* dmax) -> hyb_status {
    launch_cg_dir_stats(g, S->d, nu, part, m->st);
    HYB_LAUNCHED(m);
    launch_sum(part, kReduceBlocks, scal + 2, m->st);
    HYB_LAUNCHED(m);
    launch_max(part + kReduceBlocks, kReduceBlocks, scal + 3, m->st);
    HYB_LAUNCHED(m);
    HYB_CU(cudaMemcpyAsync(m->hscal + 2, scal + 2, 2 * sizeof(double), cudaMemcpyDeviceToHost, m->st));
    HYB_CU(cudaStreamSynchronize(m->st));
    *dJ0 = m->hscal[2];
    *dmax = m->hscal[3];
    return HYB_OK;
  };
  double dJ0 = 0.0, dmax = 0.0;
  HYB_TRY(dir_stats(&dJ0, &dmax));
  if (dJ0 >= 0.0) {  // not a descent direction: restart
    beta = 0.0;
    launch_cg_direction(g, a, P->a_min, P->a_max, vol, 0.0, S->d, nu, m->st);
    HYB_LAUNCHED(m);
    HYB_TRY(dir_stats(&dJ0, &dmax));
  }
  // Step length: parabola through F(0), F'(0) and a trial F(alpha_t); the
  // trial is the previous step unless that step did not lower F.
  const bool reseed = S->iter == 0 || !(S->alpha > 0.0) || !(J0 < S->J);
  const double at = reseed ? 0.5 / std::max(dmax, 1e-300) : S->alpha;
  double* atr = (double*)m->atrial.p;
  launch_cg_axpy_clip(a, S->d, at, P->a_min, P->a_max, P->a0, atr, nu, part, m->st);
  HYB_LAUNCHED(m);
  launch_sum(part, kReduceBlocks, scal + 4, m->st);
  HYB_LAUNCHED(m);
  HYB_TRY(forward_impl<T>(m, atr, src, nsrc, nsteps, dt, tr, false));
  double Jtd = 0.0;
  HYB_TRY(misfit_impl<T>(m, tr, obs, P->weights, &Jtd, nullptr));
  HYB_CU(cudaMemcpyAsync(m->hscal + 4, scal + 4, sizeof(double), cudaMemcpyDeviceToHost, m->st));
  HYB_CU(cudaStreamSynchronize(m->st));
  const double Jt = Jtd + 0.5 * P->gamma * vol * m->hscal[4];
  const double alpha = quadratic_step(J0, dJ0, at, Jt);
  launch_cg_axpy_clip(a, S->d, alpha, P->a_min, P->a_max, P->a0, a, nu, part, m->st);
  HYB_LAUNCHED(m);
  S->gnorm2 = gpn2;
  S->alpha = alpha;
  S->J = J0;
  S->iter += 1;
  if (R) {
    R->J = J0;
    R->J_data = Jd;
    R->gnorm = std::sqrt(gn2);
    R->gpnorm = std::sqrt(gpn2);
    R->alpha = alpha;
    R->beta = beta;
    R->dJ0 = dJ0;
    R->alpha_trial = at;
    R->J_trial = Jt;
  }
  return HYB_OK;
}

hyb_status check_sources(const hyb_mesh* m, const hyb_source* src, int nsrc) {
  if (!src) return fail(HYB_ERR_ARG, "null source array");
  if (nsrc < 1 || nsrc > kMaxSlots) return fail(HYB_ERR_ARG, "n_src must be in [1, %d]", kMaxSlots);
  for (int s = 0; s < nsrc; ++s) {
    if (src[s].face < 0 || src[s].face > 5) return fail(HYB_ERR_ARG, "source %d: bad face %d", s, src[s].face);
    if (!(src[s].omega > 0.0)) return fail(HYB_ERR_ARG, "source %d: omega must be > 0", s);
    for (int a = 0; a < 3; ++a)
      if (!std::isfinite(src[s].dir[a])) return fail(HYB_ERR_ARG, "source %d: direction is not finite", s);
  }
  (void)m;
  return HYB_OK;
}

hyb_status check_time(const hyb_mesh* m, int nsteps, double dt) {
  if (nsteps < 1) return fail(HYB_ERR_ARG, "nsteps must be >= 1");
  if (!(dt > 0.0)) return fail(HYB_ERR_ARG, "dt must be > 0");
  const double dt_max = m->dt_max;
  if (dt > dt_max * (1.0 + 1e-12))
    return fail(HYB_ERR_CFL, "dt = %.17g exceeds the stability bound dt_max = %.17g", dt, dt_max);
  return HYB_OK;
}

}  // namespace

extern "C" {

const char* hyb_last_error(void) { return g_err.c_str(); }

hyb_status hyb_mesh_create(const hyb_mesh_desc* d, void* stream, hyb_mesh** out) {
  if (!d || !out) return fail(HYB_ERR_ARG, "null argument");
  *out = nullptr;
  for (int a = 0; a < 3; ++a)
    if (d->n[a] < 3) return fail(HYB_ERR_ARG, "n[%d] = %d must be >= 3", a, d->n[a]);
  if ((long long)d->n[0] * d->n[1] >= (1LL << 31)) return fail(HYB_ERR_ARG, "lattice plane too large");
  const bool spaced = d->spacing[0] != 0.0 || d->spacing[1] != 0.0 || d->spacing[2] != 0.0;
  if (!spaced && !(d->h > 0.0)) return fail(HYB_ERR_ARG, "h must be > 0");
  if (d->precision != HYB_FP64 && d->precision != HYB_FP32) return fail(HYB_ERR_ARG, "bad precision");
  if (d->ckpt_every < 0) return fail(HYB_ERR_ARG, "ckpt_every must be >= 0");
  if (d->wait_cycles < HYB_WAIT_NONE) return fail(HYB_ERR_ARG, "wait_cycles must be >= 0 or HYB_WAIT_NONE");
  if (d->adjoint_mode != HYB_ADJ_EXACT && d->adjoint_mode != HYB_ADJ_PAPER) return fail(HYB_ERR_ARG, "bad adjoint_mode");
  if (d->fem_path != HYB_FEM_STENCIL && d->fem_path != HYB_FEM_TET_ALL) return fail(HYB_ERR_ARG, "bad fem_path");
  if (d->fem_path == HYB_FEM_TET_ALL && d->refine_mask)
    return fail(HYB_ERR_ARG, "fem_path HYB_FEM_TET_ALL takes no refinement");
  if (d->model != HYB_MODEL_WAVE && d->model != HYB_MODEL_TELEGRAPH) return fail(HYB_ERR_ARG, "bad model");
  if (d->model == HYB_MODEL_TELEGRAPH) {
    if (d->refine_mask || d->adjoint_mode != HYB_ADJ_EXACT || d->fem_path != HYB_FEM_STENCIL)
      return fail(HYB_ERR_ARG, "the telegraph model takes no refinement, the exact adjoint and the stencil path");
    for (int a = 0; a < 3; ++a)
      if (d->fem_lo[a] < 2 || d->fem_hi[a] > d->n[a] - 3)
        return fail(HYB_ERR_ARG, "the telegraph model needs 2 <= fem_lo and fem_hi <= n - 3 on every axis");
  }
  if (!(d->a_max > 0.0)) return fail(HYB_ERR_ARG, "a_max must be > 0");
  for (int a = 0; spaced && a < 3; ++a)
    if (!(d->spacing[a] > 0.0 && d->spacing[a] < 1e300))
      return fail(HYB_ERR_ARG, "spacing[%d] must be > 0 (or all three 0)", a);
  const bool ani = spaced && !(d->spacing[0] == d->spacing[1] && d->spacing[1] == d->spacing[2]);
  if (ani && (d->refine_mask || d->adjoint_mode != HYB_ADJ_EXACT || d->model != HYB_MODEL_WAVE))
    return fail(HYB_ERR_ARG, "per-axis steps take no refinement, the exact adjoint and the wave model");
  for (int f = 0; f < 6; ++f)
    if (d->bc[f] != HYB_BC_NEUMANN0 && d->bc[f] != HYB_BC_ABC) return fail(HYB_ERR_ARG, "bad bc[%d]", f);
  const bool fem = d->fem_lo[0] >= 0;
  if (fem) {
    for (int a = 0; a < 3; ++a) {
      if (d->fem_lo[a] < 0 || d->fem_hi[a] > d->n[a] - 1 || d->fem_hi[a] - d->fem_lo[a] < 2)
        return fail(HYB_ERR_ARG, "FEM block axis %d: need 0 <= lo, hi <= n-1, hi - lo >= 2", a);
    }
  }
  hyb_mesh* m = new (std::nothrow) hyb_mesh();
  if (!m) return fail(HYB_ERR_OOM, "host allocation failed");
  m->d = *d;
  if (spaced) m->d.h = d->spacing[0];  // equal steps: the isotropic lattice of that step
  m->ani = ani;
  for (int a = 0; a < 3; ++a) m->hv[a] = spaced ? d->spacing[a] : d->h;
  m->st = (cudaStream_t)stream;
  for (int a = 0; a < 3; ++a) m->n[a] = d->n[a];
  m->N = (long long)d->n[0] * d->n[1] * d->n[2];
  m->px = (d->n[0] + 7) & ~7;  // rows start on 32-byte boundaries (whole sectors per warp row)
  m->Np = (long long)m->px * d->n[1] * d->n[2];
  m->fem = fem;
  for (int a = 0; a < 3; ++a) {
    if (fem) {
      m->fl[a] = d->fem_lo[a] + 1;
      m->fh[a] = d->fem_hi[a] - 1;
      m->fn[a] = m->fh[a] - m->fl[a] + 1;
      m->wl[a] = d->fem_lo[a];
      m->wn[a] = d->fem_hi[a] - d->fem_lo[a] + 1;
      m->un[a] = d->fem_hi[a] - d->fem_lo[a] - 2;
    } else {
      m->fl[a] = 1;
      m->fh[a] = 0;
      m->fn[a] = 0;
      m->wl[a] = 0;
      m->wn[a] = 0;
      m->un[a] = 0;
    }
  }
  if (fem) {
    m->wx0 = m->wl[0] & ~3;
    m->wpx = (m->wl[0] + m->wn[0] - m->wx0 + 3) & ~3;
    m->hx0 = m->fl[0] & ~7;
    m->hpx = (m->fh[0] + 1 - m->hx0 + 7) & ~7;
  }
  m->wsz = (long long)m->wpx * m->wn[1] * m->wn[2];
  m->nu = (long long)m->un[0] * m->un[1] * m->un[2];
  m->nown = (long long)m->fn[0] * m->fn[1] * m->fn[2];
  m->hbox = (long long)m->hpx * m->fn[1] * m->fn[2];
  m->obs_stride = std::max(d->n[0] * d->n[1], std::max(d->n[0] * d->n[2], d->n[1] * d->n[2]));
  for (int f = 0; f < 6; ++f)
    if (d->bc[f] == HYB_BC_ABC) m->abc_mask |= 1 << f;
  if (ani)  // tau^2 a sum_ax 4 / dx_ax^2 <= 4: the 7-point row's bound (Eq. (CFL) for equal steps)
    m->dt_max = 1.0 / std::sqrt(d->a_max * (1.0 / (m->hv[0] * m->hv[0]) + 1.0 / (m->hv[1] * m->hv[1]) +
                                            1.0 / (m->hv[2] * m->hv[2])));
  else
    m->dt_max = m->d.h / std::sqrt(3.0 * d->a_max);
  hyb_status st = HYB_OK;
  if (fem) st = ensure(m, m->W, 3 * (size_t)m->wsz * esize(m));
  if (st == HYB_OK) st = ensure(m, m->flag, 2 * sizeof(int));
  if (st == HYB_OK && cudaMallocHost(&m->hscal, (16 + kMaxSlots) * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    m->hscal = nullptr;
    st = fail(HYB_ERR_OOM, "cudaMallocHost failed");
  }
  if (st == HYB_OK && cudaMemsetAsync(m->flag.p, 0, 2 * sizeof(int), m->st) != cudaSuccess)
    st = fail(HYB_ERR_CUDA, "cudaMemsetAsync failed");
  if (st == HYB_OK && cudaStreamCreateWithFlags(&m->cap, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    st = fail(HYB_ERR_CUDA, "stream creation failed");
  }
  if (st == HYB_OK) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&m->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      st = fail(HYB_ERR_CUDA, "device query failed");
    } else {
      m->bps = std::min(step_blocks_per_sm(d->precision, 0), step_blocks_per_sm(d->precision, 1));
    }
  }
  if (st == HYB_OK && d->fem_path == HYB_FEM_TET_ALL) st = build_kuhn(m);
  if (st == HYB_OK && d->refine_mask && fem && m->nu > 0) {
    if (d->n[0] < 5 || d->n[1] < 5 || d->n[2] < 5) st = fail(HYB_ERR_ARG, "refinement needs >= 5 nodes per axis");
    else st = build_refined(m, d->refine_mask);
  }
  if (st != HYB_OK) {
    hyb_mesh_destroy(m);
    return st;
  }
  *out = m;
  return HYB_OK;
}

hyb_status hyb_mesh_query(const hyb_mesh* m, hyb_mesh_info* o) {
  if (!m || !o) return fail(HYB_ERR_ARG, "null argument");
  o->n_nodes = m->N;
  o->n_unknown = m->nu;
  o->n_fem_owned = m->nown;
  for (int a = 0; a < 3; ++a) o->unknown_dims[a] = m->un[a];
  o->obs_stride = m->obs_stride;
  o->dt_max = m->dt_max;
  o->n_centres = m->nc;
  o->n_sparse_rows = m->nr;
  o->n_sparse_nnz = m->nnz;
  o->voxel_volume = cell_volume(m);
  o->device_bytes = m->bytes;
  o->launches = m->launches;
  return HYB_OK;
}

hyb_status hyb_mesh_destroy(hyb_mesh* m) {
  if (!m) return HYB_OK;
  cudaStreamSynchronize(m->st);
  DevBuf* bufs[] = {&m->W, &m->G, &m->flag, &m->U, &m->L, &m->hist, &m->ckpt, &m->part, &m->scal,
                    &m->g, &m->atrial, &m->cot, &m->trace, &m->rmask, &m->rzr, &m->refvox, &m->refvox_id,
                    &m->k9, &m->rcid, &m->avox, &m->rpos, &m->rvxyz, &m->sdamp, &m->ones,
                    &m->CU, &m->CL, &m->chist, &m->cckpt, &m->I0, &m->IC0, &m->acopy, &m->kuhn, &m->kuhn_v};
  for (DevBuf* b : bufs) release(*b);
  for (auto& dir : m->items)
    for (DevBuf& b : dir) release(b);
  if (m->hscal) cudaFreeHost(m->hscal);
  for (SweepGraph& g : m->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  if (m->cap) cudaStreamDestroy(m->cap);
  delete m;
  return HYB_OK;
}

hyb_status hyb_set_stream(hyb_mesh* m, void* stream) {
  if (!m) return fail(HYB_ERR_ARG, "null mesh");
  m->st = (cudaStream_t)stream;
  return HYB_OK;
}

hyb_status hyb_forward(hyb_mesh* m, const double* a, const hyb_source* src, int32_t n_src, int32_t nsteps,
                       double dt, void* trace) {
  if (!m || !trace) return fail(HYB_ERR_ARG, "null argument");
  if (m->nu > 0 && !a) return fail(HYB_ERR_ARG, "null coefficient");
  HYB_TRY(check_sources(m, src, n_src));
  HYB_TRY(check_time(m, nsteps, dt));
  if (m->d.precision == HYB_FP64)
    return forward_impl<double>(m, a, src, n_src, nsteps, dt, (double*)trace, true);
  return forward_impl<float>(m, a, src, n_src, nsteps, dt, (float*)trace, true);
}

hyb_status hyb_set_initial(hyb_mesh* m, const void* u0, const void* u_prev, const void* c0, const void* c_prev) {
  if (!m) return fail(HYB_ERR_ARG, "null mesh");
  if (!u0) {
    m->have_init = false;
    return HYB_OK;
  }
  if (!u_prev) return fail(HYB_ERR_ARG, "u_prev is needed with u0");
  const size_t es = esize(m), fb = (size_t)m->Np * es, cb = (size_t)m->nc * es;
  HYB_TRY(ensure(m, m->I0, 2 * fb));
  HYB_TRY(ensure(m, m->IC0, 2 * cb));
  HYB_CU(cudaMemsetAsync(m->I0.p, 0, 2 * fb, m->st));
  const void* lv[2] = {u0, u_prev};
  for (int q = 0; q < 2; ++q)
    HYB_CU(cudaMemcpy2DAsync((char*)m->I0.p + q * fb, (size_t)m->px * es, lv[q], (size_t)m->n[0] * es,
                             (size_t)m->n[0] * es, (size_t)m->n[1] * m->n[2], cudaMemcpyDeviceToDevice, m->st));
  if (m->nc) {
    const void* cv[2] = {c0, c_prev};
    for (int q = 0; q < 2; ++q) {
      if (cv[q]) HYB_CU(cudaMemcpyAsync((char*)m->IC0.p + q * cb, cv[q], cb, cudaMemcpyDeviceToDevice, m->st));
      else HYB_CU(cudaMemsetAsync((char*)m->IC0.p + q * cb, 0, cb, m->st));
    }
  }
  m->have_init = true;
  return HYB_OK;
}

hyb_status hyb_forward_batch(hyb_mesh* m, const double* a, const hyb_source* src, int32_t n_src, int32_t nsteps,
                             double dt, void* trace) {
  if (!m || !trace) return fail(HYB_ERR_ARG, "null argument");
  if (m->nu > 0 && !a) return fail(HYB_ERR_ARG, "null coefficient");
  if (m->d.fem_path == HYB_FEM_TET_ALL) return fail(HYB_ERR_ARG, "no batches on the HYB_FEM_TET_ALL path");
  if (m->d.model == HYB_MODEL_TELEGRAPH) return fail(HYB_ERR_ARG, "no batches with the telegraph model");
  if (m->ani) return fail(HYB_ERR_ARG, "no batches with per-axis steps");
  HYB_TRY(check_sources(m, src, n_src));
  HYB_TRY(check_time(m, nsteps, dt));
  if (m->d.precision == HYB_FP64)
    return forward_impl<double>(m, a, src, n_src, nsteps, dt, (double*)trace, true, true);
  return forward_impl<float>(m, a, src, n_src, nsteps, dt, (float*)trace, true, true);
}

hyb_status hyb_misfit_batch(hyb_mesh* m, const void* trace, const void* u_obs, int32_t weights, double* J_host,
                            void* cot) {
  if (!m || !trace || !u_obs) return fail(HYB_ERR_ARG, "null argument");
  if (weights != HYB_WEIGHTS_PLAIN && weights != HYB_WEIGHTS_QUADRATURE) return fail(HYB_ERR_ARG, "bad weights");
  if (m->d.precision == HYB_FP64)
    return misfit_batch_impl<double>(m, (const double*)trace, (const double*)u_obs, weights, J_host, (double*)cot);
  return misfit_batch_impl<float>(m, (const float*)trace, (const float*)u_obs, weights, J_host, (float*)cot);
}

hyb_status hyb_gradient_batch(hyb_mesh* m, const double* a, double gamma, double a0, double* g_out) {
  if (!m) return fail(HYB_ERR_ARG, "null mesh");
  if (m->nu > 0 && (!a || !g_out)) return fail(HYB_ERR_ARG, "null coefficient or output");
  if (!m->have_adj) return fail(HYB_ERR_STATE, "hyb_gradient_batch needs a preceding hyb_adjoint");
  if (!m->batch) return fail(HYB_ERR_STATE, "hyb_gradient_batch needs a preceding hyb_forward_batch");
  if (m->nu == 0) return HYB_OK;
  for (int s = 0; s < m->nsrc; ++s) {
    launch_grad_finalize((const double*)m->G.p + (size_t)s * m->nu, 1, a + (size_t)s * m->nu, grad_scale(m), gamma,
                         cell_volume(m), a0, g_out + (size_t)s * m->nu, m->nu, m->st);
    HYB_LAUNCHED(m);
  }
  return HYB_OK;
}

hyb_status hyb_adjoint(hyb_mesh* m, const void* cot, int32_t accumulate) {
  if (!m || !cot) return fail(HYB_ERR_ARG, "null argument");
  if (m->d.precision == HYB_FP64) return adjoint_impl<double>(m, (const double*)cot, accumulate);
  return adjoint_impl<float>(m, (const float*)cot, accumulate);
}

hyb_status hyb_gradient(hyb_mesh* m, const double* a, double gamma, double a0, double* g_out) {
  if (!m) return fail(HYB_ERR_ARG, "null mesh");
  if (m->nu > 0 && (!a || !g_out)) return fail(HYB_ERR_ARG, "null coefficient or output");
  if (!m->have_adj) return fail(HYB_ERR_STATE, "hyb_gradient needs a preceding hyb_adjoint");
  if (m->batch) return fail(HYB_ERR_STATE, "the last forward was a batch: use hyb_gradient_batch");
  if (m->nu == 0) return HYB_OK;
  launch_grad_finalize((const double*)m->G.p, m->nsrc, a, grad_scale(m), gamma, cell_volume(m), a0, g_out, m->nu,
                       m->st);
  HYB_LAUNCHED(m);
  return HYB_OK;
}

hyb_status hyb_misfit(hyb_mesh* m, const void* trace, const void* u_obs, int32_t weights, double* J_host,
                      void* cot) {
  if (!m || !trace || !u_obs) return fail(HYB_ERR_ARG, "null argument");
  if (weights != HYB_WEIGHTS_PLAIN && weights != HYB_WEIGHTS_QUADRATURE) return fail(HYB_ERR_ARG, "bad weights");
  if (m->d.precision == HYB_FP64)
    return misfit_impl<double>(m, (const double*)trace, (const double*)u_obs, weights, J_host, (double*)cot);
  return misfit_impl<float>(m, (const float*)trace, (const float*)u_obs, weights, J_host, (float*)cot);
}

hyb_status hyb_cg_step(hyb_mesh* m, double* a, const void* u_obs, const hyb_source* src, int32_t n_src,
                       int32_t nsteps, double dt, const hyb_cg_params* p, hyb_cg_state* s, hyb_cg_report* r) {
  if (!m || !a || !u_obs || !p || !s || !s->d) return fail(HYB_ERR_ARG, "null argument");
  if (m->nu == 0) return fail(HYB_ERR_ARG, "the mesh has no unknown voxels");
  if (!(p->a_min <= p->a_max) || p->a_max > m->d.a_max * (1.0 + 1e-12))
    return fail(HYB_ERR_ARG, "need a_min <= a_max <= the mesh's a_max");
  if (p->weights != HYB_WEIGHTS_PLAIN && p->weights != HYB_WEIGHTS_QUADRATURE) return fail(HYB_ERR_ARG, "bad weights");
  HYB_TRY(check_sources(m, src, n_src));
  HYB_TRY(check_time(m, nsteps, dt));
  if (m->d.precision == HYB_FP64)
    return cg_impl<double>(m, a, (const double*)u_obs, src, n_src, nsteps, dt, p, s, r);
  return cg_impl<float>(m, a, (const float*)u_obs, src, n_src, nsteps, dt, p, s, r);
}

hyb_status hyb_get_field(hyb_mesh* m, int32_t which, int32_t isrc, void* out) {
  if (!m || !out) return fail(HYB_ERR_ARG, "null argument");
  if (!m->have_run || isrc < 0 || isrc >= m->nsrc) return fail(HYB_ERR_STATE, "no such field");
  const size_t fb = (size_t)m->Np * esize(m);
  const char* src = nullptr;
  const int r_u_last = ((m->nsteps % 3) + 3) % 3;
  const int r_u_prev = (((m->nsteps - 1) % 3) + 3) % 3;
  if ((which == HYB_FIELD_U_LAST || which == HYB_FIELD_U_PREV) && !m->u_levels)
    return fail(HYB_ERR_STATE, "a checkpointed adjoint has reused the forward's levels: read u before hyb_adjoint");
  if (which == HYB_FIELD_U_LAST) {
    src = (const char*)m->U.p + ((size_t)r_u_last * m->nsrc + isrc) * fb;
  } else if (which == HYB_FIELD_U_PREV) {
    src = (const char*)m->U.p + ((size_t)r_u_prev * m->nsrc + isrc) * fb;
  } else if (which == HYB_FIELD_LAMBDA_FIRST) {
    if (!m->have_adj) return fail(HYB_ERR_STATE, "no adjoint has run");
    const size_t lv = m->d.adjoint_mode == HYB_ADJ_PAPER ? 0 : 1;  // lambda^0 (paper) or lambda^1
    src = (const char*)m->L.p + (lv * m->nsrc + isrc) * fb;
  } else {
    return fail(HYB_ERR_ARG, "bad field selector");
  }
  const size_t es = esize(m);  // drop the row padding
  HYB_CU(cudaMemcpy2DAsync(out, (size_t)m->n[0] * es, src, (size_t)m->px * es, (size_t)m->n[0] * es,
                           (size_t)m->n[1] * m->n[2], cudaMemcpyDeviceToDevice, m->st));
  return HYB_OK;
}

hyb_status hyb_misfit_noalloc(const void* trace, const void* u_obs, int32_t precision, int32_t n_src,
                              int32_t nsteps, int32_t obs_stride, const int32_t* face_dims, double dt, double h,
                              int32_t weights, double* J_dev, void* cot, void* stream) {
  if (!trace || !u_obs || !face_dims || !J_dev) return fail(HYB_ERR_ARG, "null argument");
  if (precision != HYB_FP64 && precision != HYB_FP32) return fail(HYB_ERR_ARG, "bad precision");
  if (weights != HYB_WEIGHTS_PLAIN && weights != HYB_WEIGHTS_QUADRATURE) return fail(HYB_ERR_ARG, "bad weights");
  if (n_src < 1 || n_src > kMaxSlots) return fail(HYB_ERR_ARG, "n_src must be in [1, %d]", kMaxSlots);
  if (nsteps < 0 || obs_stride < 1) return fail(HYB_ERR_ARG, "bad nsteps or obs_stride");
  // bound the size factor by factor, before forming the product
  const long long cap = noalloc_max_entries();
  if ((long long)nsteps + 1 > cap / obs_stride / n_src)
    return fail(HYB_ERR_ARG, "trace of %d x %lld x %d entries exceeds the %lld entries hyb_misfit_noalloc can reduce",
                n_src, (long long)nsteps + 1, obs_stride, cap);
  const long long total = (long long)n_src * ((long long)nsteps + 1) * obs_stride;
  MisfitGeom g;
  std::memset(&g, 0, sizeof g);
  g.n_src = n_src;
  g.nsteps = nsteps;
  g.stride = obs_stride;
  for (int s = 0; s < n_src; ++s) {
    g.np[s] = face_dims[2 * s];
    g.nq[s] = face_dims[2 * s + 1];
    if (g.np[s] < 1 || g.nq[s] < 1 || (long long)g.np[s] * g.nq[s] > obs_stride)
      return fail(HYB_ERR_ARG, "source %d: face dims do not fit obs_stride", s);
  }
  const bool quad = weights == HYB_WEIGHTS_QUADRATURE;
  g.wt = quad ? dt : 1.0;
  for (int s = 0; s < n_src; ++s) g.hh[s] = quad ? h * h : 1.0;
  g.halve = quad ? 1 : 0;
  double* scratch = nullptr;
  HYB_CU(noalloc_scratch(&scratch));
  const cudaStream_t st = (cudaStream_t)stream;
  if (precision == HYB_FP64)
    launch_misfit_noalloc<double>(g, (const double*)trace, (const double*)u_obs, (double*)cot, scratch, total,
                                  J_dev, st);
  else
    launch_misfit_noalloc<float>(g, (const float*)trace, (const float*)u_obs, (float*)cot, scratch, total, J_dev,
                                 st);
  HYB_CU(cudaGetLastError());
  return HYB_OK;
}

hyb_status hyb_sync(hyb_mesh* m) {
  if (!m) return fail(HYB_ERR_ARG, "null mesh");
  // stream-ordered copies only: other streams (other meshes) keep running
  int* flag = (int*)(m->hscal + 14);
  HYB_CU(cudaMemcpyAsync(flag, m->flag.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, m->st));
  HYB_CU(cudaStreamSynchronize(m->st));
  if (flag[0] || flag[1]) {
    const int f0 = flag[0];
    HYB_CU(cudaMemsetAsync(m->flag.p, 0, 2 * sizeof(int), m->st));
    HYB_CU(cudaStreamSynchronize(m->st));
    if (f0) return fail(HYB_ERR_CFL, "a coefficient value exceeded a_max (or was not finite)");
    return fail(HYB_ERR_TIMEOUT, "a step kernel's bounded wait for its staged planes ran out");
  }
  return HYB_OK;
}

}  // extern "C"
