// Training and evaluation kernels of the learned troubled-cell gate
// (24 -> 32 -> 32 -> 1, ReLU, sigmoid output), on BF16 tensor cores with FP32
// accumulation (mma.sync m16n8k16), and their C ABI (include/gks2l.h).
//
// k_mlp_grad: forward and backward of the logistic loss
//   L = sum_i pos_w y_i softplus(-s_i) + (1 - y_i) softplus(s_i)
// over a batch; each warp takes 16 samples at a time. Layer outputs stay in
// registers and are reused as the A operand of the next product; the weight
// gradients dW = dZ^T H are products over the batch dimension, read
// transposed from a per-warp shared-memory tile. Sums are FP32, in a fixed
// order (per-warp partials, then a reduction in warp order): the gradient is
// the same from run to run.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "gks2l.h"
#include "mlp.cuh"

using namespace gks2l;

namespace {

constexpr int TPB = 128;

__device__ __forceinline__ unsigned pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  __nv_bfloat162 v;
  v.x = lo;
  v.y = hi;
  return *reinterpret_cast<unsigned *>(&v);
}
__device__ __forceinline__ float bfr(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float softplus(float x) { return x > 0.f ? x + log1pf(expf(-x)) : log1pf(expf(x)); }
__device__ __forceinline__ float sigm(float x) { return 1.f / (1.f + expf(-x)); }

struct WarpTiles {
  __nv_bfloat16 X[16 * 32], H1[16 * 32], DZ2[16 * 32], DZ1[16 * 32];
};

// A fragment of T^T (m = column of T, k = row of T) from a bf16 [16][32] tile
__device__ __forceinline__ void load_a_t(unsigned a[4], const __nv_bfloat16 *T, int m0, int lane) {
  const int g = lane >> 2, c = (lane & 3) * 2;
  a[0] = pack2(T[c * 32 + m0 + g], T[(c + 1) * 32 + m0 + g]);
  a[1] = pack2(T[c * 32 + m0 + g + 8], T[(c + 1) * 32 + m0 + g + 8]);
  a[2] = pack2(T[(c + 8) * 32 + m0 + g], T[(c + 9) * 32 + m0 + g]);
  a[3] = pack2(T[(c + 8) * 32 + m0 + g + 8], T[(c + 9) * 32 + m0 + g + 8]);
}
// B fragment (k = row of T, n = column of T) from a bf16 [16][32] tile
__device__ __forceinline__ void load_b_t(unsigned b[2], const __nv_bfloat16 *T, int n0, int lane) {
  const int g = lane >> 2, c = (lane & 3) * 2;
  b[0] = pack2(T[c * 32 + n0 + g], T[(c + 1) * 32 + n0 + g]);
  b[1] = pack2(T[(c + 8) * 32 + n0 + g], T[(c + 9) * 32 + n0 + g]);
}

// Each warp writes its partial sums (NTRAIN gradients, then the loss) to
// part[warp]; k_mlp_reduce adds them up in warp order, so the result does not
// depend on scheduling.
constexpr int NPART = MLP_NTRAIN + 1;

__global__ void __launch_bounds__(TPB) k_mlp_grad(const float *X, const float *y, int n, const float *P, float pos_w,
                                                  float *part) {
  __shared__ MlpDev w;
  __shared__ WarpTiles tiles[TPB / 32];
  mlp_pack(w, P, 0.f, threadIdx.x, TPB);
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int g = lane >> 2, c = (lane & 3) * 2;
  WarpTiles &S = tiles[wid];
  float gW1[2][4][4], gW2[2][4][4];
  float gb1[4][2], gb2[4][2], gw3[4][2], gb3 = 0.f, lsum = 0.f;
  for (int a = 0; a < 2; a++)
    for (int b = 0; b < 4; b++)
      for (int i = 0; i < 4; i++) gW1[a][b][i] = gW2[a][b][i] = 0.f;
  for (int b = 0; b < 4; b++)
    for (int i = 0; i < 2; i++) gb1[b][i] = gb2[b][i] = gw3[b][i] = 0.f;
  const int ntile = (n + 15) / 16;
  for (int t = blockIdx.x * (TPB / 32) + wid; t < ntile; t += gridDim.x * (TPB / 32)) {
    const int r0 = t * 16;
    for (int i = lane; i < 16 * 32; i += 32) {
      int r = i >> 5, k = i & 31, row = r0 + r;
      float v = 0.f;
      if (k < MLP_IN && row < n) v = (X[(size_t)row * MLP_IN + k] - w.mean[k]) * w.istd[k];
      S.X[i] = __float2bfloat16_rn(v);
    }
    __syncwarp();
    // ---- forward
    float z1[4][4];
    for (int nt = 0; nt < 4; nt++)
      for (int i = 0; i < 4; i++) z1[nt][i] = 0.f;
    for (int ks = 0; ks < 2; ks++) {
      unsigned a[4];
      load_a(a, S.X, 32, 0, 16 * ks, lane);
      for (int nt = 0; nt < 4; nt++) {
        unsigned b[2];
        load_b_nk(b, w.w1, 32, 8 * nt, 16 * ks, lane);
        mma_bf16(z1[nt], a, b);
      }
    }
    unsigned a2[2][4];
    float m1[4][4];
    for (int nt = 0; nt < 4; nt++) {
      int col = 8 * nt + c;
      float p[4] = {z1[nt][0] + w.b1[col], z1[nt][1] + w.b1[col + 1], z1[nt][2] + w.b1[col], z1[nt][3] + w.b1[col + 1]};
      float h[4];
      for (int i = 0; i < 4; i++) {
        m1[nt][i] = p[i] > 0.f ? 1.f : 0.f;
        h[i] = fmaxf(p[i], 0.f);
      }
      a2[nt >> 1][2 * (nt & 1)] = pack_bf16(h[0], h[1]);
      a2[nt >> 1][2 * (nt & 1) + 1] = pack_bf16(h[2], h[3]);
      S.H1[g * 32 + col] = __float2bfloat16_rn(h[0]);
      S.H1[g * 32 + col + 1] = __float2bfloat16_rn(h[1]);
      S.H1[(g + 8) * 32 + col] = __float2bfloat16_rn(h[2]);
      S.H1[(g + 8) * 32 + col + 1] = __float2bfloat16_rn(h[3]);
    }
    float z2[4][4];
    for (int nt = 0; nt < 4; nt++)
      for (int i = 0; i < 4; i++) z2[nt][i] = 0.f;
    for (int ks = 0; ks < 2; ks++)
      for (int nt = 0; nt < 4; nt++) {
        unsigned b[2];
        load_b_nk(b, w.w2, 32, 8 * nt, 16 * ks, lane);
        mma_bf16(z2[nt], a2[ks], b);
      }
    float h2v[4][4], m2[4][4];
    float s0 = 0.f, s1 = 0.f;
    for (int nt = 0; nt < 4; nt++) {
      int col = 8 * nt + c;
      float p[4] = {z2[nt][0] + w.b2[col], z2[nt][1] + w.b2[col + 1], z2[nt][2] + w.b2[col], z2[nt][3] + w.b2[col + 1]};
      for (int i = 0; i < 4; i++) {
        m2[nt][i] = p[i] > 0.f ? 1.f : 0.f;
        h2v[nt][i] = bfr(fmaxf(p[i], 0.f));
      }
      s0 += h2v[nt][0] * w.w3[col] + h2v[nt][1] * w.w3[col + 1];
      s1 += h2v[nt][2] * w.w3[col] + h2v[nt][3] * w.w3[col + 1];
    }
    s0 += __shfl_xor_sync(0xffffffffu, s0, 1);
    s0 += __shfl_xor_sync(0xffffffffu, s0, 2);
    s1 += __shfl_xor_sync(0xffffffffu, s1, 1);
    s1 += __shfl_xor_sync(0xffffffffu, s1, 2);
    s0 += w.b3;
    s1 += w.b3;
    // ---- loss and its derivative in the logit, rows g and g + 8
    const int ra = r0 + g, rb = r0 + g + 8;
    const bool va = ra < n, vb = rb < n;
    const float ya = va ? y[ra] : 0.f, yb = vb ? y[rb] : 0.f;
    const float dsa = va ? (-pos_w * ya * sigm(-s0) + (1.f - ya) * sigm(s0)) : 0.f;
    const float dsb = vb ? (-pos_w * yb * sigm(-s1) + (1.f - yb) * sigm(s1)) : 0.f;
    if ((lane & 3) == 0) {
      if (va) lsum += pos_w * ya * softplus(-s0) + (1.f - ya) * softplus(s0);
      if (vb) lsum += pos_w * yb * softplus(-s1) + (1.f - yb) * softplus(s1);
      gb3 += dsa + dsb;
    }
    // ---- backward
    float dz2[4][4];
    unsigned ad[2][4];
    for (int nt = 0; nt < 4; nt++) {
      int col = 8 * nt + c;
      dz2[nt][0] = dsa * w.w3[col] * m2[nt][0];
      dz2[nt][1] = dsa * w.w3[col + 1] * m2[nt][1];
      dz2[nt][2] = dsb * w.w3[col] * m2[nt][2];
      dz2[nt][3] = dsb * w.w3[col + 1] * m2[nt][3];
      gw3[nt][0] += dsa * h2v[nt][0] + dsb * h2v[nt][2];
      gw3[nt][1] += dsa * h2v[nt][1] + dsb * h2v[nt][3];
      gb2[nt][0] += dz2[nt][0] + dz2[nt][2];
      gb2[nt][1] += dz2[nt][1] + dz2[nt][3];
      ad[nt >> 1][2 * (nt & 1)] = pack_bf16(dz2[nt][0], dz2[nt][1]);
      ad[nt >> 1][2 * (nt & 1) + 1] = pack_bf16(dz2[nt][2], dz2[nt][3]);
      S.DZ2[g * 32 + col] = __float2bfloat16_rn(dz2[nt][0]);
      S.DZ2[g * 32 + col + 1] = __float2bfloat16_rn(dz2[nt][1]);
      S.DZ2[(g + 8) * 32 + col] = __float2bfloat16_rn(dz2[nt][2]);
      S.DZ2[(g + 8) * 32 + col + 1] = __float2bfloat16_rn(dz2[nt][3]);
    }
    // dH1 = dZ2 W2: B element (k = out, n = in) = W2[k][n]
    float dh1[4][4];
    for (int nt = 0; nt < 4; nt++)
      for (int i = 0; i < 4; i++) dh1[nt][i] = 0.f;
    for (int ks = 0; ks < 2; ks++)
      for (int nt = 0; nt < 4; nt++) {
        const int k0 = 16 * ks + c, n0 = 8 * nt + g;
        unsigned b[2] = {pack2(w.w2[k0 * 32 + n0], w.w2[(k0 + 1) * 32 + n0]),
                         pack2(w.w2[(k0 + 8) * 32 + n0], w.w2[(k0 + 9) * 32 + n0])};
        mma_bf16(dh1[nt], ad[ks], b);
      }
    for (int nt = 0; nt < 4; nt++) {
      int col = 8 * nt + c;
      float d[4];
      for (int i = 0; i < 4; i++) d[i] = dh1[nt][i] * m1[nt][i];
      gb1[nt][0] += d[0] + d[2];
      gb1[nt][1] += d[1] + d[3];
      S.DZ1[g * 32 + col] = __float2bfloat16_rn(d[0]);
      S.DZ1[g * 32 + col + 1] = __float2bfloat16_rn(d[1]);
      S.DZ1[(g + 8) * 32 + col] = __float2bfloat16_rn(d[2]);
      S.DZ1[(g + 8) * 32 + col + 1] = __float2bfloat16_rn(d[3]);
    }
    __syncwarp();
    // weight gradients over the 16 samples: dW2 = dZ2^T H1, dW1 = dZ1^T X
    for (int mt = 0; mt < 2; mt++) {
      unsigned a[4], a1[4];
      load_a_t(a, S.DZ2, 16 * mt, lane);
      load_a_t(a1, S.DZ1, 16 * mt, lane);
      for (int nt = 0; nt < 4; nt++) {
        unsigned b[2], b1[2];
        load_b_t(b, S.H1, 8 * nt, lane);
        mma_bf16(gW2[mt][nt], a, b);
        load_b_t(b1, S.X, 8 * nt, lane);
        mma_bf16(gW1[mt][nt], a1, b1);
      }
    }
    __syncwarp();
  }
  // reduce the per-lane column partials over the eight row groups
  for (int nt = 0; nt < 4; nt++)
    for (int i = 0; i < 2; i++)
      for (int o = 4; o < 32; o <<= 1) {
        gb1[nt][i] += __shfl_xor_sync(0xffffffffu, gb1[nt][i], o);
        gb2[nt][i] += __shfl_xor_sync(0xffffffffu, gb2[nt][i], o);
        gw3[nt][i] += __shfl_xor_sync(0xffffffffu, gw3[nt][i], o);
      }
  for (int o = 1; o < 32; o <<= 1) {
    gb3 += __shfl_xor_sync(0xffffffffu, gb3, o);
    lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  }
  float *out = part + (size_t)(blockIdx.x * (TPB / 32) + wid) * NPART;
  if (lane < 4) {
    for (int nt = 0; nt < 4; nt++)
      for (int i = 0; i < 2; i++) {
        int col = 8 * nt + c + i;
        out[MLP_B1 + col] = gb1[nt][i];
        out[MLP_B2 + col] = gb2[nt][i];
        out[MLP_W3 + col] = gw3[nt][i];
      }
  }
  if (lane == 0) {
    out[MLP_B3] = gb3;
    out[MLP_NTRAIN] = lsum;
  }
  for (int mt = 0; mt < 2; mt++)
    for (int nt = 0; nt < 4; nt++)
      for (int i = 0; i < 4; i++) {
        int o = 16 * mt + g + (i >= 2 ? 8 : 0), in = 8 * nt + c + (i & 1);
        out[MLP_W2 + o * MLP_H + in] = gW2[mt][nt][i];
        if (in < MLP_IN) out[MLP_W1 + o * MLP_IN + in] = gW1[mt][nt][i];
      }
}

__global__ void k_mlp_reduce(const float *part, int nparts, float *grads, float *loss_out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NPART) return;
  float s = 0.f;
  for (int w = 0; w < nparts; w++) s += part[(size_t)w * NPART + i];
  if (i < MLP_NTRAIN) grads[i] = s;
  else *loss_out = s;
}

__global__ void k_mlp_adam(float *P, const float *G, float *M, float *V, int n, int step, float lr, float scale) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  float gr = G[i] * scale;
  float m = b1 * M[i] + (1.f - b1) * gr;
  float v = b2 * V[i] + (1.f - b2) * gr * gr;
  M[i] = m;
  V[i] = v;
  float mh = m / (1.f - powf(b1, (float)step)), vh = v / (1.f - powf(b2, (float)step));
  P[i] -= lr * mh / (sqrtf(vh) + eps);
}

// logits with the inference image (normalisation folded into layer 1), the
// network the reconstruction runs
__global__ void __launch_bounds__(TPB) k_mlp_forward(const float *X, int n, const float *P, float *logits) {
  constexpr int LD = 40;   // padded row stride of the feature tiles (bank spread)
  __shared__ MlpDev w;
  __shared__ __align__(16) __nv_bfloat16 Xs[TPB / 32][32 * LD];
  mlp_pack_folded(w, P, 0.f, threadIdx.x, TPB);
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  MlpFrags F;
  mlp_frags(F, w, lane);
  const int ntile = (n + 31) / 32;
  for (int t = blockIdx.x * (TPB / 32) + wid; t < ntile; t += gridDim.x * (TPB / 32)) {
    const int r0 = t * 32;
    for (int i = lane; i < 32 * 32; i += 32) {
      int r = i >> 5, k = i & 31, row = r0 + r;
      float v = 0.f;
      if (k < MLP_IN && row < n) v = X[(size_t)row * MLP_IN + k];
      Xs[wid][r * LD + k] = __float2bfloat16_rn(v);
    }
    __syncwarp();
    float s = mlp_tile32(F, Xs[wid], LD, lane);
    if (r0 + lane < n) logits[r0 + lane] = s;
    __syncwarp();
  }
}

unsigned grid_for(int n, int per_block, int cap) {
  int b = (n + per_block - 1) / per_block;
  return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

extern "C" int gks2l_mlp_grad(const float *d_X, const float *d_y, int32_t n, const float *d_params, float pos_weight,
                              float *d_grads, float *d_loss, void *stream) {
  if (n <= 0 || !d_X || !d_y || !d_params || !d_grads || !d_loss) return GKS2L_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  // a few blocks per SM: each warp loops over 16-sample tiles
  const unsigned grid = grid_for(n, 16 * (TPB / 32), 608);
  const int nparts = (int)grid * (TPB / 32);
  float *part = nullptr;
  if (cudaMallocAsync((void **)&part, (size_t)nparts * NPART * sizeof(float), s) != cudaSuccess) return GKS2L_ECUDA;
  k_mlp_grad<<<grid, TPB, 0, s>>>(d_X, d_y, n, d_params, pos_weight, part);
  k_mlp_reduce<<<(NPART + 255) / 256, 256, 0, s>>>(part, nparts, d_grads, d_loss);
  const bool ok = cudaGetLastError() == cudaSuccess;
  if (cudaFreeAsync(part, s) != cudaSuccess || !ok) return GKS2L_ECUDA;
  return GKS2L_OK;
}

extern "C" int gks2l_mlp_adam(float *d_params, const float *d_grads, float *d_m, float *d_v, int32_t step, float lr,
                              float scale, void *stream) {
  if (!d_params || !d_grads || !d_m || !d_v || step <= 0) return GKS2L_EINVAL;
  k_mlp_adam<<<(MLP_NTRAIN + 255) / 256, 256, 0, (cudaStream_t)stream>>>(d_params, d_grads, d_m, d_v, MLP_NTRAIN,
                                                                          step, lr, scale);
  return cudaGetLastError() == cudaSuccess ? GKS2L_OK : GKS2L_ECUDA;
}

extern "C" int gks2l_mlp_forward(const float *d_X, int32_t n, const float *d_params, float *d_logits, void *stream) {
  if (n <= 0 || !d_X || !d_params || !d_logits) return GKS2L_EINVAL;
  k_mlp_forward<<<grid_for(n, 32 * (TPB / 32), 4096), TPB, 0, (cudaStream_t)stream>>>(d_X, n, d_params, d_logits);
  return cudaGetLastError() == cudaSuccess ? GKS2L_OK : GKS2L_ECUDA;
}
