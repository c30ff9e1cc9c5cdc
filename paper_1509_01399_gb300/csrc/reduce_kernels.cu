// FP64 reductions and vector updates of the optimisation layer: the data
// misfit of the Tikhonov functional (Eq. (functional)) with the adjoint's
// cotangent, the gradient of Eq. (gradient1) plus the Tikhonov term, and the
// conjugate-gradient vectors of Algorithm 3.  Every reduction runs on a
// fixed grid of kReduceBlocks blocks followed by a one-block pass, so the
// summation order (and the result) does not depend on timing.
#include <cfloat>

#include "hyb_internal.h"

namespace hyb {
namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide sum for blockDim.x a multiple of 32 (<= 1024); result in thread 0.
__device__ double block_sum(double v) {
  __shared__ double sh[32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (w == 0) v = warp_sum(v);
  __syncthreads();
  return v;
}

__device__ double block_max(double v) {
  __shared__ double sh[32];
  v = warp_max(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  v = (threadIdx.x < nw) ? sh[threadIdx.x] : -DBL_MAX;
  if (w == 0) v = warp_max(v);
  __syncthreads();
  return v;
}

template <typename T>
__global__ void __launch_bounds__(kReduceThreads) misfit_kernel(const MisfitGeom g, const T* __restrict__ trace,
                                                                const T* __restrict__ obs, T* __restrict__ cot,
                                                                double* __restrict__ partials) {
  const long long rows = (long long)g.n_src * (g.nsteps + 1);
  const long long total = rows * g.stride;
  double acc = 0.0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int jj = (int)(e % g.stride);
    const long long r = e / g.stride;
    const int k = (int)(r % (g.nsteps + 1));
    const int s = (int)(r / (g.nsteps + 1));
    const int np = g.np[s], nq = g.nq[s];
    T cv = T(0);
    if (k >= 1 && jj < np * nq) {
      double m = g.hh[s];
      if (g.halve) {
        const int cp = jj % np, cq = jj / np;
        if (cp == 0 || cp == np - 1) m *= 0.5;
        if (cq == 0 || cq == nq - 1) m *= 0.5;
      }
      const double d = (double)trace[e] - (double)obs[e];
      const double w = g.wt * m;
      acc += 0.5 * w * d * d;
      cv = (T)(w * d);
    }
    if (cot) cot[e] = cv;
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

__global__ void sum_kernel(const double* __restrict__ p, int n, double* out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += p[i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) *out = acc;
}

__global__ void max_kernel(const double* __restrict__ p, int n, double* out) {
  double acc = -DBL_MAX;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc = fmax(acc, p[i]);
  acc = block_max(acc);
  if (threadIdx.x == 0) *out = acc;
}

__global__ void grad_finalize_kernel(const double* __restrict__ G, int n_src, const double* __restrict__ a,
                                     double scale, double gamma, double vol, double a0,
                                     double* __restrict__ g, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < n_src; ++q) s += G[(long long)q * n + i];
    g[i] = scale * s + gamma * vol * (a[i] - a0);
  }
}

// a at a bound of [lo, hi] with v pointing out of it
__device__ __forceinline__ bool blocked(double a, double v, double lo, double hi) {
  return (a <= lo && v < 0.0) || (a >= hi && v > 0.0);
}

__global__ void __launch_bounds__(kReduceThreads) cg_norms_kernel(const double* __restrict__ g,
                                                                  const double* __restrict__ a, double a0,
                                                                  double lo, double hi, long long n,
                                                                  double* __restrict__ partials) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double gi = g[i];
    s0 += gi * gi;
    const double e = a[i] - a0;
    s1 += e * e;
    // descent moves a along -g: a component whose -g leaves [lo, hi] is clipped
    if (!blocked(a[i], -gi, lo, hi)) s2 += gi * gi;
  }
  s0 = block_sum(s0);
  s1 = block_sum(s1);
  s2 = block_sum(s2);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = s0;
    partials[gridDim.x + blockIdx.x] = s1;
    partials[2 * gridDim.x + blockIdx.x] = s2;
  }
}

__global__ void cg_direction_kernel(const double* __restrict__ g, const double* __restrict__ a, double lo,
                                    double hi, double vol, double beta, double* __restrict__ d, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double ai = a[i];
    const double gl = blocked(ai, -g[i], lo, hi) ? 0.0 : g[i] / vol;
    const double v = beta != 0.0 ? -gl + beta * d[i] : -gl;
    d[i] = blocked(ai, v, lo, hi) ? 0.0 : v;
  }
}

__global__ void __launch_bounds__(kReduceThreads) cg_dir_stats_kernel(const double* __restrict__ g,
                                                                      const double* __restrict__ d, long long n,
                                                                      double* __restrict__ partials) {
  double s = 0.0, m = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    s += g[i] * d[i];
    m = fmax(m, fabs(d[i]));
  }
  s = block_sum(s);
  m = block_max(m);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = s;
    partials[gridDim.x + blockIdx.x] = m;
  }
}

__global__ void __launch_bounds__(kReduceThreads) cg_axpy_clip_kernel(
    const double* __restrict__ a, const double* __restrict__ d, double alpha, double lo, double hi,
    double a0, double* out, long long n, double* __restrict__ partials) {
  double s = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double v = fmin(fmax(a[i] + alpha * d[i], lo), hi);
    out[i] = v;
    const double e = v - a0;
    s += e * e;
  }
  s = block_sum(s);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

}  // namespace

template <typename T>
void launch_misfit(const MisfitGeom& g, const T* trace, const T* obs, T* cot, double* partials,
                   cudaStream_t st) {
  misfit_kernel<T><<<kReduceBlocks, kReduceThreads, 0, st>>>(g, trace, obs, cot, partials);
}
template void launch_misfit<float>(const MisfitGeom&, const float*, const float*, float*, double*,
                                   cudaStream_t);
template void launch_misfit<double>(const MisfitGeom&, const double*, const double*, double*, double*,
                                    cudaStream_t);

void launch_sum(const double* partials, int n, double* out, cudaStream_t st) {
  sum_kernel<<<1, 256, 0, st>>>(partials, n, out);
}

void launch_max(const double* partials, int n, double* out, cudaStream_t st) {
  max_kernel<<<1, 256, 0, st>>>(partials, n, out);
}

void launch_grad_finalize(const double* G, int n_src, const double* a, double scale, double gamma,
                          double vol, double a0, double* g, long long n, cudaStream_t st) {
  if (n == 0) return;
  grad_finalize_kernel<<<kReduceBlocks, kReduceThreads, 0, st>>>(G, n_src, a, scale, gamma, vol, a0, g, n);
}

void launch_cg_norms(const double* g, const double* a, double a0, double lo, double hi, long long n,
                     double* partials, cudaStream_t st) {
  cg_norms_kernel<<<kReduceBlocks, kReduceThreads, 0, st>>>(g, a, a0, lo, hi, n, partials);
}

void launch_cg_direction(const double* g, const double* a, double lo, double hi, double vol, double beta,
                         double* d, long long n, cudaStream_t st) {
  if (n == 0) return;
  cg_direction_kernel<<<kReduceBlocks, kReduceThreads, 0, st>>>(g, a, lo, hi, vol, beta, d, n);
}

void launch_cg_dir_stats(const double* g, const double* d, long long n, double* partials,
                         cudaStream_t st) {
  cg_dir_stats_kernel<<<kReduceBlocks, kReduceThreads, 0, st>>>(g, d, n, partials);
}

void launch_cg_axpy_clip(const double* a, const double* d, double alpha, double lo, double hi,
                         double a0, double* out, long long n, double* partials, cudaStream_t st) {
  cg_axpy_clip_kernel<<<kReduceBlocks, kReduceThreads, 0, st>>>(a, d, alpha, lo, hi, a0, out, n, partials);
}

}  // namespace hyb

// ---------------------------------------------------------------------------
// Allocation-free variant of the misfit reduction (hyb_misfit_noalloc).
//
// Some callers cannot allocate device memory at the point where they need
// the misfit: code running while a stream is being captured into a CUDA
// graph, latency-critical loops in which cudaMalloc (which can synchronise
// the whole device) is forbidden, or hosts that hand all device memory out
// of their own fixed pool.  This entry point needs no mesh and no
// workspace: its per-block partial sums live in the file-scope array below,
// reserved once on every GPU that loads the library and kept until the
// process exits.
// ---------------------------------------------------------------------------
#include <mutex>

namespace hyb {
namespace {

constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocPerThread = 16;
constexpr long long kNoAllocChunk = (long long)kNoAllocThreads * kNoAllocPerThread;  // entries per block
constexpr int kNoAllocSlots = 16384;  // partial sums: 128 KiB per device

__device__ __align__(256) double g_noalloc_partials[kNoAllocSlots];

template <typename T>
__global__ void __launch_bounds__(kNoAllocThreads) misfit_chunk_kernel(const hyb::MisfitGeom g,
                                                                       const T* __restrict__ trace,
                                                                       const T* __restrict__ obs,
                                                                       T* __restrict__ cot,
                                                                       double* __restrict__ partials,
                                                                       long long total) {
  const long long base = (long long)blockIdx.x * kNoAllocChunk;
  double acc = 0.0;
  for (int q = 0; q < kNoAllocPerThread; ++q) {
    const long long e = base + (long long)q * kNoAllocThreads + threadIdx.x;
    if (e >= total) break;
    const int jj = (int)(e % g.stride);
    const long long r = e / g.stride;
    const int k = (int)(r % (g.nsteps + 1));
    const int s = (int)(r / (g.nsteps + 1));
    const int np = g.np[s], nq = g.nq[s];
    T cv = T(0);
    if (k >= 1 && jj < np * nq) {
      double m = g.hh[s];
      if (g.halve) {
        const int cp = jj % np, cq = jj / np;
        if (cp == 0 || cp == np - 1) m *= 0.5;
        if (cq == 0 || cq == nq - 1) m *= 0.5;
      }
      const double d = (double)trace[e] - (double)obs[e];
      const double w = g.wt * m;
      acc += 0.5 * w * d * d;
      cv = (T)(w * d);
    }
    if (cot) cot[e] = cv;
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

__global__ void noalloc_sum_kernel(const double* __restrict__ p, int n, double* out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += p[i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) *out = acc;
}

std::mutex g_noalloc_mu;
double* g_noalloc_ptr[256] = {nullptr};

}  // namespace

long long noalloc_max_entries() { return kNoAllocChunk * kNoAllocSlots; }

// Device address of the partials array on the current device, looked up once
// per device (the host-side symbol is not a device address).
cudaError_t noalloc_scratch(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = (double*)p;
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

template <typename T>
void launch_misfit_noalloc(const MisfitGeom& g, const T* trace, const T* obs, T* cot, double* scratch,
                           long long total, double* J_dev, cudaStream_t st) {
  const int blocks = (int)((total + kNoAllocChunk - 1) / kNoAllocChunk);
  if (blocks > 0) misfit_chunk_kernel<T><<<blocks, kNoAllocThreads, 0, st>>>(g, trace, obs, cot, scratch, total);
  noalloc_sum_kernel<<<1, 256, 0, st>>>(scratch, blocks, J_dev);
}
template void launch_misfit_noalloc<float>(const MisfitGeom&, const float*, const float*, float*, double*,
                                           long long, double*, cudaStream_t);
template void launch_misfit_noalloc<double>(const MisfitGeom&, const double*, const double*, double*, double*,
                                            long long, double*, cudaStream_t);

}  // namespace hyb
