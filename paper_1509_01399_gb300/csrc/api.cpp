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
  const void* io = nullptr;
  int accumulate = 0;
  int nsteps = 0, nsrc = 0;
  double dt = 0.0;
  int face[16] = {0};
  double omega[16] = {0.0}, amp[16] = {0.0};
  const void* bufs[8] = {nullptr};
};

bool same_key(const SweepKey& a, const SweepKey& b) {
  if (a.kind != b.kind || a.io != b.io || a.accumulate != b.accumulate || a.nsteps != b.nsteps ||
      a.nsrc != b.nsrc || a.dt != b.dt)
    return false;
  for (int i = 0; i < a.nsrc; ++i)
    if (a.face[i] != b.face[i] || a.omega[i] != b.omega[i] || a.amp[i] != b.amp[i]) return false;
  for (int i = 0; i < 8; ++i)
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
  long long N = 0;
  bool fem = false;
  int fl[3], fh[3], fn[3], wl[3], wn[3], un[3];
  long long wsz = 0, nu = 0, nown = 0;
  int obs_stride = 0;
  int abc_mask = 0;
  DevBuf W, G, flag, U, L, hist, ckpt, part, scal, g, atrial, cot, trace;
  double* hscal = nullptr;  // pinned host copy of device scalars
  bool have_fwd = false;    // the adjoint has what it needs
  bool have_run = false;    // a forward has run (time grid known)
  bool have_adj = false;
  int nsteps = 0, nsrc = 0;
  double dt = 0.0;
  hyb_source src[kMaxSlots];
  long long launches = 0;
  long long bytes = 0;
  cudaStream_t cap = nullptr;  // private stream used only to capture sweep graphs
  cudaStream_t aux = nullptr;  // runs the boundary-shell kernel of each step
  cudaEvent_t ev_bulk = nullptr, ev_shell = nullptr;
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
  k.io = io;
  k.accumulate = accumulate;
  k.nsteps = nsteps;
  k.nsrc = nsrc;
  k.dt = dt;
  for (int i = 0; i < nsrc; ++i) {
    k.face[i] = src[i].face;
    k.omega[i] = src[i].omega;
    k.amp[i] = src[i].amp;
  }
  const void* b[8] = {m->U.p, m->L.p, m->hist.p, m->ckpt.p, m->G.p, m->W.p, nullptr, nullptr};
  for (int i = 0; i < 8; ++i) k.bufs[i] = b[i];
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

// Boundary state of the step leaving t_k = k dt for one source: the source
// face carries the Neumann flux p(t_k) = amp sin(omega t_k) while
// t_k <= 2 pi / omega (Eq. (f), Model Problem 2) and otherwise takes the
// mesh's own condition.
void phase_of(const hyb_mesh* m, const hyb_source& s, int k, double dt, int* mask, int* srcf,
              double* p) {
  const double t = k * dt;
  if (t <= 2.0 * M_PI / s.omega) {
    *mask = m->abc_mask & ~(1 << s.face);
    *srcf = s.face;
    *p = s.amp * std::sin(s.omega * t);
  } else {
    *mask = m->abc_mask;
    *srcf = -1;
    *p = 0.0;
  }
}

int mask_at(const hyb_mesh* m, const hyb_source& s, int k, double dt) {
  int mask, f;
  double p;
  phase_of(m, s, k, dt, &mask, &f, &p);
  return mask;
}

// Launch geometry of one step: the interior kernel covers nodes 1 .. n-2 on
// every axis in 32 x 8 tiles and z chunks; the edge kernel the nodes within
// one node of two faces.  Lattices with fewer than 5 nodes on an axis use a
// single generic kernel instead.
void step_geometry(const hyb_mesh* m, int nslots, int* npb, int* ntx, int* zchunk, int* nzc, int* small,
                   int* nedge) {
  *small = (m->n[0] < 5 || m->n[1] < 5 || m->n[2] < 5) ? 1 : 0;
  *nedge = *small ? 0 : 1 + (m->n[0] - 4 + 7) / 8 + (m->n[1] - 4 + 7) / 8 + (m->n[2] - 4 + 7) / 8;
  const long long bx = m->n[0] - 2, by = m->n[1] - 2, bz = m->n[2] - 2;
  *ntx = (int)((bx + kTileX - 1) / kTileX);
  const int nty = (int)((by + kTileY - 1) / kTileY);
  *npb = *ntx * nty;
  const long long target = 152LL * 8;  // resident blocks wanted on 152 SMs
  const long long per_z = (long long)(*npb) * nslots;
  long long want = (target + per_z - 1) / per_z;
  if (want < 1) want = 1;
  long long z = (bz + want - 1) / want;
  z = std::max<long long>(z, 2);
  z = std::min<long long>(z, bz);
  *zchunk = (int)z;
  *nzc = (int)((bz + z - 1) / z);
}

// One time level on two streams: the interior kernel on `st`, the edge
// kernel on the mesh's aux stream.  Each waits for both kernels of the
// previous level (fork/join through two events), so they overlap with each
// other but not across levels.  begin_steps/join_steps bracket a run of
// levels; other work on `st` must come after join_steps.
hyb_status begin_steps(hyb_mesh* m, cudaStream_t st) {
  HYB_CU(cudaEventRecord(m->ev_bulk, st));
  HYB_CU(cudaEventRecord(m->ev_shell, st));
  return HYB_OK;
}

template <class Bulk, class Shell>
hyb_status step_pair(hyb_mesh* m, cudaStream_t st, Bulk bulk, Shell shell) {
  HYB_CU(cudaStreamWaitEvent(m->aux, m->ev_bulk, 0));
  HYB_CU(cudaStreamWaitEvent(st, m->ev_shell, 0));
  bulk(st);
  HYB_LAUNCHED(m);
  HYB_CU(cudaEventRecord(m->ev_bulk, st));
  shell(m->aux);
  HYB_LAUNCHED(m);
  HYB_CU(cudaEventRecord(m->ev_shell, m->aux));
  return HYB_OK;
}

hyb_status join_steps(hyb_mesh* m, cudaStream_t st) {
  HYB_CU(cudaStreamWaitEvent(st, m->ev_shell, 0));
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
  A.W = (const T*)m->W.p;
  A.G = (double*)m->G.p;
  const double h = m->d.h;
  A.c2 = (T)(dt * dt / (h * h));
  A.r = (T)((h - dt) / (h + dt));
  step_geometry(m, nslots, &A.npb, &A.ntx, &A.zchunk, &A.nzc, &A.small, &A.nedge);
  A.nslots = nslots;
}

template <typename T>
T* field_buf(const hyb_mesh* m, const DevBuf& b, int nsrc, int s, int level) {
  const int r = ((level % 3) + 3) % 3;
  return (T*)b.p + ((size_t)r * nsrc + s) * (size_t)m->N;
}

// Fill the forward slots of step k (u^k -> u^{k+1}).
template <typename T>
void forward_slots(const hyb_mesh* m, StepArgs<T>& A, const hyb_source* src, int nsrc, int nsteps,
                   double dt, int k, T* trace, T* hist_level) {
  for (int s = 0; s < nsrc; ++s) {
    Slot<T>& S = A.s[s];
    S.cur = field_buf<T>(m, m->U, nsrc, s, k);
    S.prev = field_buf<T>(m, m->U, nsrc, s, k - 1);
    S.next = field_buf<T>(m, m->U, nsrc, s, k + 1);
    S.obs_w = trace ? trace + ((size_t)s * (nsteps + 1) + (k + 1)) * (size_t)m->obs_stride : nullptr;
    S.obs_r = nullptr;
    S.hist_w = hist_level ? hist_level + (size_t)s * m->nown : nullptr;
    S.hist_r = nullptr;
    int mask, f;
    double p;
    phase_of(m, src[s], k, dt, &mask, &f, &p);
    S.mask_f = mask;
    S.mask_e = 0;
    S.mask_c = 0;
    S.src_face = f;
    S.srcval = (T)(dt * dt * 2.0 * p / m->d.h);
    S.obs_face = src[s].face;
  }
}

template <typename T>
hyb_status forward_impl(hyb_mesh* m, const double* a, const hyb_source* src, int nsrc, int nsteps,
                        double dt, T* trace, bool keep) {
  const size_t fb = (size_t)m->N * sizeof(T);
  const int C = m->d.ckpt_every;
  const bool ckpt = C > 0;
  HYB_TRY(ensure(m, m->U, 3 * (size_t)nsrc * fb));
  if (keep && m->nown > 0) {
    if (!ckpt) {
      HYB_TRY(ensure(m, m->hist, (size_t)nsteps * nsrc * m->nown * sizeof(T)));
    } else {
      const size_t nseg = ((size_t)nsteps + C - 1) / C;
      HYB_TRY(ensure(m, m->ckpt, nseg * 2 * (size_t)nsrc * fb));
      HYB_TRY(ensure(m, m->hist, (size_t)C * nsrc * m->nown * sizeof(T)));
    }
  }
  StepArgs<T> A;
  base_args(m, A, dt, nsrc);
  if (m->fem) {
    launch_set_coef<T>(A, (T*)m->W.p, a, m->d.a_max, (int*)m->flag.p, m->st);
    HYB_LAUNCHED(m);
  }
  auto body = [&](cudaStream_t st) -> hyb_status {
    for (int s = 0; s < nsrc; ++s) {
      HYB_CU(cudaMemsetAsync(field_buf<T>(m, m->U, nsrc, s, 0), 0, fb, st));
      HYB_CU(cudaMemsetAsync(field_buf<T>(m, m->U, nsrc, s, -1), 0, fb, st));
    }
    if (trace) HYB_CU(cudaMemsetAsync(trace, 0, (size_t)nsrc * (nsteps + 1) * m->obs_stride * sizeof(T), st));
    T* hist = (T*)m->hist.p;
    if (keep && !ckpt && m->nown > 0) HYB_CU(cudaMemsetAsync(hist, 0, (size_t)nsrc * m->nown * sizeof(T), st));
    const size_t lvl = (size_t)nsrc * m->nown;
    HYB_TRY(begin_steps(m, st));
    for (int k = 0; k < nsteps; ++k) {
      if (keep && ckpt && m->nown > 0 && k > 0 && k % C == 0) {
        HYB_TRY(join_steps(m, st));
        const size_t seg = (size_t)(k / C);
        for (int s = 0; s < nsrc; ++s) {
          char* base = (char*)m->ckpt.p + ((seg * nsrc + s) * 2) * fb;
          HYB_CU(cudaMemcpyAsync(base, field_buf<T>(m, m->U, nsrc, s, k), fb, cudaMemcpyDeviceToDevice, st));
          HYB_CU(cudaMemcpyAsync(base + fb, field_buf<T>(m, m->U, nsrc, s, k - 1), fb, cudaMemcpyDeviceToDevice,
                                 st));
        }
        HYB_TRY(begin_steps(m, st));
      }
      T* hl = (keep && !ckpt && m->nown > 0 && k + 1 <= nsteps - 1) ? hist + (size_t)(k + 1) * lvl : nullptr;
      forward_slots<T>(m, A, src, nsrc, nsteps, dt, k, trace, hl);
      HYB_TRY(step_pair(m, st, [&](cudaStream_t q) { launch_forward_bulk<T>(A, q); },
                        [&](cudaStream_t q) { launch_forward_shell<T>(A, q); }));
    }
    HYB_TRY(join_steps(m, st));
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
  return HYB_OK;
}

template <typename T>
void adjoint_slots(const hyb_mesh* m, StepArgs<T>& A, const T* cot, int j, const T* hist_level) {
  const int nsrc = m->nsrc, nsteps = m->nsteps;
  for (int s = 0; s < nsrc; ++s) {
    Slot<T>& S = A.s[s];
    S.cur = field_buf<T>(m, m->L, nsrc, s, j + 1);
    S.prev = field_buf<T>(m, m->L, nsrc, s, j + 2);
    S.next = field_buf<T>(m, m->L, nsrc, s, j);
    S.obs_w = nullptr;
    S.obs_r = cot + ((size_t)s * (nsteps + 1) + j) * (size_t)m->obs_stride;
    S.hist_w = nullptr;
    S.hist_r = hist_level ? hist_level + (size_t)s * m->nown : nullptr;
    S.srcval = T(0);
    S.src_face = -1;
    S.mask_f = mask_at(m, m->src[s], j, m->dt);
    S.mask_e = mask_at(m, m->src[s], j - 1, m->dt);
    S.mask_c = mask_at(m, m->src[s], j + 1, m->dt);
    S.obs_face = m->src[s].face;
  }
}

template <typename T>
hyb_status pair_first(hyb_mesh* m, StepArgs<T>& A, const T* level0, cudaStream_t st) {
  for (int s = 0; s < m->nsrc; ++s) {
    StepArgs<T> B = A;
    B.G = (double*)m->G.p + (size_t)s * m->nu;
    launch_pair<T>(B, level0 + (size_t)s * m->nown, field_buf<T>(m, m->L, m->nsrc, s, 1), st);
    HYB_LAUNCHED(m);
  }
  return HYB_OK;
}

template <typename T>
hyb_status adjoint_impl(hyb_mesh* m, const T* cot, int accumulate) {
  if (!m->have_fwd) return fail(HYB_ERR_STATE, "hyb_adjoint needs a preceding hyb_forward of this mesh");
  const int nsrc = m->nsrc, nsteps = m->nsteps;
  const double dt = m->dt;
  const size_t fb = (size_t)m->N * sizeof(T);
  const int C = m->d.ckpt_every;
  const bool ckpt = C > 0;
  HYB_TRY(ensure(m, m->L, 3 * (size_t)nsrc * fb));
  HYB_TRY(ensure(m, m->G, (size_t)nsrc * m->nu * sizeof(double)));
  StepArgs<T> A;   // adjoint steps
  base_args(m, A, dt, nsrc);
  StepArgs<T> F;   // recomputed forward steps
  base_args(m, F, dt, nsrc);
  auto body = [&](cudaStream_t st) -> hyb_status {
    if (!accumulate) HYB_CU(cudaMemsetAsync(m->G.p, 0, (size_t)nsrc * m->nu * sizeof(double), st));
    for (int s = 0; s < nsrc; ++s) {
      HYB_CU(cudaMemsetAsync(field_buf<T>(m, m->L, nsrc, s, nsteps + 1), 0, fb, st));
      HYB_CU(cudaMemsetAsync(field_buf<T>(m, m->L, nsrc, s, nsteps + 2), 0, fb, st));
    }
    T* hist = (T*)m->hist.p;
    const size_t lvl = (size_t)nsrc * m->nown;
    const bool pairing = m->nu > 0 && m->nown > 0;
    auto adj_step = [&](int j, const T* hl) -> hyb_status {
      adjoint_slots<T>(m, A, cot, j, hl);
      return step_pair(m, st, [&](cudaStream_t q) { launch_adjoint_bulk<T>(A, q); },
                       [&](cudaStream_t q) { launch_adjoint_shell<T>(A, q); });
    };
    auto fwd_step = [&](int k, T* hl) -> hyb_status {
      forward_slots<T>(m, F, m->src, nsrc, nsteps, dt, k, nullptr, hl);
      return step_pair(m, st, [&](cudaStream_t q) { launch_forward_bulk<T>(F, q); },
                       [&](cudaStream_t q) { launch_forward_shell<T>(F, q); });
    };
    HYB_TRY(begin_steps(m, st));
    if (!ckpt) {
      for (int j = nsteps; j >= 1; --j) {
        const T* hl = (pairing && j <= nsteps - 1) ? hist + (size_t)j * lvl : nullptr;
        HYB_TRY(adj_step(j, hl));
      }
      HYB_TRY(join_steps(m, st));
      if (pairing) HYB_TRY(pair_first<T>(m, A, hist, st));
      return HYB_OK;
    }
    HYB_TRY(adj_step(nsteps, nullptr));
    const int nseg = (nsteps + C - 1) / C;
    for (int seg = nseg - 1; seg >= 0; --seg) {
      const int kb = seg * C;
      const int ke = std::min((seg + 1) * C, nsteps) - 1;
      if (pairing) {
        HYB_TRY(join_steps(m, st));
        for (int s = 0; s < nsrc; ++s) {
          T* u0 = field_buf<T>(m, m->U, nsrc, s, kb);
          T* um = field_buf<T>(m, m->U, nsrc, s, kb - 1);
          if (seg == 0) {
            HYB_CU(cudaMemsetAsync(u0, 0, fb, st));
            HYB_CU(cudaMemsetAsync(um, 0, fb, st));
          } else {
            const char* base = (const char*)m->ckpt.p + (((size_t)seg * nsrc + s) * 2) * fb;
            HYB_CU(cudaMemcpyAsync(u0, base, fb, cudaMemcpyDeviceToDevice, st));
            HYB_CU(cudaMemcpyAsync(um, base + fb, fb, cudaMemcpyDeviceToDevice, st));
          }
          launch_extract_owned<T>(F, u0, hist + (size_t)s * m->nown, st);
          HYB_LAUNCHED(m);
        }
        HYB_TRY(begin_steps(m, st));
        for (int k = kb; k < ke; ++k) HYB_TRY(fwd_step(k, hist + (size_t)(k + 1 - kb) * lvl));
      }
      for (int j = ke; j >= std::max(kb, 1); --j)
        HYB_TRY(adj_step(j, pairing ? hist + (size_t)(j - kb) * lvl : nullptr));
    }
    HYB_TRY(join_steps(m, st));
    if (pairing) HYB_TRY(pair_first<T>(m, A, hist, st));
    return HYB_OK;
  };
  HYB_TRY(run_sweep(m, m->graphs[2], make_key(m, 2, cot, accumulate, nsteps, nsrc, dt, m->src), body));
  m->have_adj = true;
  return HYB_OK;
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
  g.hh = quad ? m->d.h * m->d.h : 1.0;
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
  const double vol = m->d.h * m->d.h * m->d.h;
  HYB_TRY(ensure(m, m->trace, tb));
  HYB_TRY(ensure(m, m->cot, tb));
  HYB_TRY(ensure(m, m->g, (size_t)nu * sizeof(double)));
  HYB_TRY(ensure(m, m->atrial, (size_t)nu * sizeof(double)));
  HYB_TRY(ensure(m, m->part, 2 * (size_t)kReduceBlocks * sizeof(double)));
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
  launch_grad_finalize((const double*)m->G.p, nsrc, a, -dt * dt / (m->d.h * m->d.h), P->gamma, vol, P->a0,
                       g, nu, m->st);
  HYB_LAUNCHED(m);
  launch_cg_norms(g, a, P->a0, nu, part, m->st);
  HYB_LAUNCHED(m);
  launch_sum(part, kReduceBlocks, scal + 0, m->st);
  HYB_LAUNCHED(m);
  launch_sum(part + kReduceBlocks, kReduceBlocks, scal + 1, m->st);
  HYB_LAUNCHED(m);
  HYB_CU(cudaMemcpyAsync(m->hscal, scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, m->st));
  HYB_CU(cudaStreamSynchronize(m->st));
  const double gn2 = m->hscal[0] / vol;  // ||g||_L2^2 with g = (dF/da) / |c|
  const double J0 = Jd + 0.5 * P->gamma * vol * m->hscal[1];
  // Step 2: Fletcher-Reeves direction.
  double beta = (S->iter > 0 && S->gnorm2 > 0.0) ? gn2 / S->gnorm2 : 0.0;
  launch_cg_direction(g, vol, beta, S->d, nu, m->st);
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
  if (dJ0 >= 0.0) {
    beta = 0.0;
    launch_cg_direction(g, vol, 0.0, S->d, nu, m->st);
    HYB_LAUNCHED(m);
    HYB_TRY(dir_stats(&dJ0, &dmax));
    dJ0 = -gn2;
  }
  // Step length: parabola through F(0), F'(0) and a trial F(alpha_t).
  const double at = S->alpha > 0.0 ? S->alpha : 0.5 / std::max(dmax, 1e-300);
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
  S->gnorm2 = gn2;
  S->alpha = alpha;
  S->iter += 1;
  if (R) {
    R->J = J0;
    R->J_data = Jd;
    R->gnorm = std::sqrt(gn2);
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
  }
  (void)m;
  return HYB_OK;
}

hyb_status check_time(const hyb_mesh* m, int nsteps, double dt) {
  if (nsteps < 1) return fail(HYB_ERR_ARG, "nsteps must be >= 1");
  if (!(dt > 0.0)) return fail(HYB_ERR_ARG, "dt must be > 0");
  const double dt_max = m->d.h / std::sqrt(3.0 * m->d.a_max);
  if (dt > dt_max * (1.0 + 1e-12))
    return fail(HYB_ERR_CFL, "dt = %.17g exceeds the CFL bound h / sqrt(3 a_max) = %.17g", dt, dt_max);
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
  if (!(d->h > 0.0)) return fail(HYB_ERR_ARG, "h must be > 0");
  if (d->precision != HYB_FP64 && d->precision != HYB_FP32) return fail(HYB_ERR_ARG, "bad precision");
  if (d->ckpt_every < 0) return fail(HYB_ERR_ARG, "ckpt_every must be >= 0");
  if (!(d->a_max > 0.0)) return fail(HYB_ERR_ARG, "a_max must be > 0");
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
  m->st = (cudaStream_t)stream;
  for (int a = 0; a < 3; ++a) m->n[a] = d->n[a];
  m->N = (long long)d->n[0] * d->n[1] * d->n[2];
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
  m->wsz = (long long)m->wn[0] * m->wn[1] * m->wn[2];
  m->nu = (long long)m->un[0] * m->un[1] * m->un[2];
  m->nown = (long long)m->fn[0] * m->fn[1] * m->fn[2];
  m->obs_stride = std::max(d->n[0] * d->n[1], std::max(d->n[0] * d->n[2], d->n[1] * d->n[2]));
  for (int f = 0; f < 6; ++f)
    if (d->bc[f] == HYB_BC_ABC) m->abc_mask |= 1 << f;
  hyb_status st = HYB_OK;
  if (fem) st = ensure(m, m->W, 3 * (size_t)m->wsz * esize(m));
  if (st == HYB_OK) st = ensure(m, m->flag, sizeof(int));
  if (st == HYB_OK && cudaMallocHost(&m->hscal, 16 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    m->hscal = nullptr;
    st = fail(HYB_ERR_OOM, "cudaMallocHost failed");
  }
  if (st == HYB_OK && cudaMemsetAsync(m->flag.p, 0, sizeof(int), m->st) != cudaSuccess)
    st = fail(HYB_ERR_CUDA, "cudaMemsetAsync failed");
  if (st == HYB_OK && (cudaStreamCreateWithFlags(&m->cap, cudaStreamNonBlocking) != cudaSuccess ||
                        cudaStreamCreateWithFlags(&m->aux, cudaStreamNonBlocking) != cudaSuccess ||
                        cudaEventCreateWithFlags(&m->ev_bulk, cudaEventDisableTiming) != cudaSuccess ||
                        cudaEventCreateWithFlags(&m->ev_shell, cudaEventDisableTiming) != cudaSuccess)) {
    cudaGetLastError();
    st = fail(HYB_ERR_CUDA, "stream or event creation failed");
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
  o->dt_max = m->d.h / std::sqrt(3.0 * m->d.a_max);
  o->voxel_volume = m->d.h * m->d.h * m->d.h;
  o->device_bytes = m->bytes;
  o->launches = m->launches;
  return HYB_OK;
}

hyb_status hyb_mesh_destroy(hyb_mesh* m) {
  if (!m) return HYB_OK;
  cudaStreamSynchronize(m->st);
  if (m->aux) cudaStreamSynchronize(m->aux);
  DevBuf* bufs[] = {&m->W, &m->G, &m->flag, &m->U, &m->L, &m->hist, &m->ckpt, &m->part, &m->scal,
                    &m->g, &m->atrial, &m->cot, &m->trace};
  for (DevBuf* b : bufs) release(*b);
  if (m->hscal) cudaFreeHost(m->hscal);
  for (SweepGraph& g : m->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  if (m->cap) cudaStreamDestroy(m->cap);
  if (m->aux) cudaStreamDestroy(m->aux);
  if (m->ev_bulk) cudaEventDestroy(m->ev_bulk);
  if (m->ev_shell) cudaEventDestroy(m->ev_shell);
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

hyb_status hyb_adjoint(hyb_mesh* m, const void* cot, int32_t accumulate) {
  if (!m || !cot) return fail(HYB_ERR_ARG, "null argument");
  if (m->d.precision == HYB_FP64) return adjoint_impl<double>(m, (const double*)cot, accumulate);
  return adjoint_impl<float>(m, (const float*)cot, accumulate);
}

hyb_status hyb_gradient(hyb_mesh* m, const double* a, double gamma, double a0, double* g_out) {
  if (!m) return fail(HYB_ERR_ARG, "null mesh");
  if (m->nu > 0 && (!a || !g_out)) return fail(HYB_ERR_ARG, "null coefficient or output");
  if (!m->have_adj) return fail(HYB_ERR_STATE, "hyb_gradient needs a preceding hyb_adjoint");
  if (m->nu == 0) return HYB_OK;
  const double h = m->d.h;
  launch_grad_finalize((const double*)m->G.p, m->nsrc, a, -m->dt * m->dt / (h * h), gamma, h * h * h, a0,
                       g_out, m->nu, m->st);
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
  const size_t fb = (size_t)m->N * esize(m);
  const char* src = nullptr;
  const int r_u_last = ((m->nsteps % 3) + 3) % 3;
  const int r_u_prev = (((m->nsteps - 1) % 3) + 3) % 3;
  if (which == HYB_FIELD_U_LAST) {
    src = (const char*)m->U.p + ((size_t)r_u_last * m->nsrc + isrc) * fb;
  } else if (which == HYB_FIELD_U_PREV) {
    src = (const char*)m->U.p + ((size_t)r_u_prev * m->nsrc + isrc) * fb;
  } else if (which == HYB_FIELD_LAMBDA_FIRST) {
    if (!m->have_adj) return fail(HYB_ERR_STATE, "no adjoint has run");
    src = (const char*)m->L.p + ((size_t)1 * m->nsrc + isrc) * fb;
  } else {
    return fail(HYB_ERR_ARG, "bad field selector");
  }
  HYB_CU(cudaMemcpyAsync(out, src, fb, cudaMemcpyDeviceToDevice, m->st));
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
  const long long total = (long long)n_src * (nsteps + 1) * obs_stride;
  if (total > noalloc_max_entries())
    return fail(HYB_ERR_ARG, "trace of %lld entries exceeds the %lld entries hyb_misfit_noalloc can reduce", total,
                noalloc_max_entries());
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
  g.hh = quad ? h * h : 1.0;
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
  HYB_CU(cudaStreamSynchronize(m->st));
  int flag = 0;
  HYB_CU(cudaMemcpy(&flag, m->flag.p, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag) {
    HYB_CU(cudaMemset(m->flag.p, 0, sizeof(int)));
    return fail(HYB_ERR_CFL, "a coefficient value exceeded a_max (or was not finite)");
  }
  return HYB_OK;
}

}  // extern "C"
