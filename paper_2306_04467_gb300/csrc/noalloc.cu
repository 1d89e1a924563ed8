// gks2l_cfl_mass_noalloc: the CFL step and per-layer mass of a state, for
// callers that cannot allocate device memory. Its scratch (one partial result
// per block) lives in a file-scope device array of fixed size; nothing is
// allocated by this entry point.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "gks2l.h"

namespace {

constexpr int kBlocks = 1024;      // partial results held in the scratch array
constexpr int kThreads = 256;

// 4 doubles per block: min(dX / U_max), sum |Omega| h1, sum |Omega| h2 and
// the number of unusable cells. Every block of a call writes its slot before
// the final pass reads it, so nothing has to start at zero.
static __device__ __align__(256) double g_noalloc_scratch[4 * kBlocks];

__device__ __forceinline__ double warp_min(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block-wide (min, sum, sum, sum) of one value per thread; result in thread 0
__device__ void block_reduce(double &r, double &m1, double &m2, double &nb) {
  __shared__ double sr[kThreads / 32], s1[kThreads / 32], s2[kThreads / 32], sb[kThreads / 32];
  r = warp_min(r);
  m1 = warp_sum(m1);
  m2 = warp_sum(m2);
  nb = warp_sum(nb);
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { sr[w] = r; s1[w] = m1; s2[w] = m2; sb[w] = nb; }
  __syncthreads();
  if (w == 0) {
    r = lane < kThreads / 32 ? sr[lane] : INFINITY;
    m1 = lane < kThreads / 32 ? s1[lane] : 0.0;
    m2 = lane < kThreads / 32 ? s2[lane] : 0.0;
    nb = lane < kThreads / 32 ? sb[lane] : 0.0;
    r = warp_min(r);
    m1 = warp_sum(m1);
    m2 = warp_sum(m2);
    nb = warp_sum(nb);
  }
}

// pass 1: per-block partials over a grid-stride range of cells
__global__ void __launch_bounds__(kThreads) k_cfl_partial(int n, const double *avg, const double *area,
                                                         const double *dX, double g, double *scratch) {
  double r = INFINITY, m1 = 0, m2 = 0, nbad = 0;
  for (int j = blockIdx.x * kThreads + threadIdx.x; j < n; j += gridDim.x * kThreads) {
    double um = 0;
    bool bad = false;
    for (int l = 0; l < 2; l++) {
      // layer l: depth at variable 3 (lower) or 0 (upper)
      int b = l == 0 ? 3 : 0;
      double h = avg[(size_t)b * n + j];
      double u = avg[(size_t)(b + 1) * n + j] / h, v = avg[(size_t)(b + 2) * n + j] / h;
      double sp = sqrt(u * u + v * v) + sqrt(g * h);
      // a non-positive depth or a non-finite speed makes the cell unusable
      // (fmax would otherwise drop a NaN speed)
      bad = bad || !(h > 0) || !isfinite(sp);
      um = fmax(um, sp);
    }
    double q = dX[j] / um;
    bad = bad || !(q > 0 && isfinite(q));
    r = fmin(r, bad ? INFINITY : q);
    nbad += bad ? 1.0 : 0.0;
    m1 += area[j] * avg[(size_t)3 * n + j];
    m2 += area[j] * avg[j];
  }
  block_reduce(r, m1, m2, nbad);
  if (threadIdx.x == 0) {
    scratch[4 * blockIdx.x] = r;
    scratch[4 * blockIdx.x + 1] = m1;
    scratch[4 * blockIdx.x + 2] = m2;
    scratch[4 * blockIdx.x + 3] = nbad;
  }
}

// pass 2: one block folds the partials and writes (dt, mass1, mass2, bad)
__global__ void __launch_bounds__(kThreads) k_cfl_final(int nb, const double *scratch, double cfl, double *out) {
  double r = INFINITY, m1 = 0, m2 = 0, nbad = 0;
  for (int b = threadIdx.x; b < nb; b += kThreads) {
    r = fmin(r, scratch[4 * b]);
    m1 += scratch[4 * b + 1];
    m2 += scratch[4 * b + 2];
    nbad += scratch[4 * b + 3];
  }
  block_reduce(r, m1, m2, nbad);
  if (threadIdx.x == 0) {
    out[0] = cfl * r;
    out[1] = m1;
    out[2] = m2;
    out[3] = nbad;
  }
}

// device address of the scratch array, looked up once per device (and kept:
// a cudaDeviceReset would make it stale, which the header rules out)
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_addr[kMaxDevices] = {nullptr};

int scratch_address(double **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GKS2L_ECUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return GKS2L_ECUDA;
    g_addr[dev] = (double *)p;
  }
  *out = g_addr[dev];
  return GKS2L_OK;
}

}  // namespace

extern "C" int gks2l_cfl_mass_noalloc(int32_t n_tri, const double *d_avg, const double *d_area,
                                      const double *d_dX, double g, double cfl, double *d_out, void *stream) {
  if (n_tri <= 0 || !d_avg || !d_area || !d_dX || !d_out || !(g > 0) || !(cfl > 0)) return GKS2L_EINVAL;
  if (n_tri > GKS2L_NOALLOC_MAX_TRI) return GKS2L_ETOOBIG;
  double *scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  int nb = (n_tri + kThreads - 1) / kThreads;
  if (nb > kBlocks) nb = kBlocks;
  k_cfl_partial<<<nb, kThreads, 0, s>>>(n_tri, d_avg, d_area, d_dX, g, scratch);
  k_cfl_final<<<1, kThreads, 0, s>>>(nb, scratch, cfl, d_out);
  return cudaGetLastError() == cudaSuccess ? GKS2L_OK : GKS2L_ECUDA;
}
