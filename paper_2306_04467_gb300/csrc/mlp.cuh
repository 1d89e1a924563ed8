// Learned troubled-cell gate: features and BF16 tensor-core MLP tiles.
//
// The gate (not part of the paper) decides per cell and stage whether the
// WENO weights of the compact reconstruction (Sec. 3.4) would depart from the
// linear ones; cells it calls smooth take the linear P3 reconstruction. The
// network is 24 -> 32 -> 32 -> 1 with ReLU hidden layers and a sigmoid output,
// BF16 weights and activations, FP32 accumulation (mma.sync m16n8k16).
#pragma once
#include <cuda_bf16.h>

#include "stage.cuh"

namespace gks2l {

constexpr int MLP_IN = 24, MLP_H = 32;
// float parameter vector: W1[32][24], b1[32], W2[32][32], b2[32], w3[32], b3,
// mean[24], inv_std[24]
constexpr int MLP_W1 = 0, MLP_B1 = MLP_W1 + MLP_H * MLP_IN, MLP_W2 = MLP_B1 + MLP_H, MLP_B2 = MLP_W2 + MLP_H * MLP_H,
              MLP_W3 = MLP_B2 + MLP_H, MLP_B3 = MLP_W3 + MLP_H, MLP_MEAN = MLP_B3 + 1, MLP_ISTD = MLP_MEAN + MLP_IN,
              MLP_NPARAM = MLP_ISTD + MLP_IN, MLP_NTRAIN = MLP_MEAN;   // trained parameters come first

// Device copy of the network: BF16 weights padded to K = 32, FP32 biases.
// A multiple of 16 bytes, so blocks copy it with 16-byte loads.
struct alignas(16) MlpDev {
  __nv_bfloat16 w1[MLP_H * 32];   // [out][in], in padded 24 -> 32 with zeros
  __nv_bfloat16 w2[MLP_H * 32];   // [out][in]
  float b1[MLP_H], b2[MLP_H], w3[MLP_H], b3;
  float mean[MLP_IN], istd[MLP_IN];
  float threshold;
};

// The 24 features of cell j: for eta1 (0-11), then h2 (12-23), over the cell
// and its three face neighbours, the deviation of the average from their
// mean and the h-scaled gradient, divided by the norm of all twelve
// (regularised by the WENO epsilon, so smooth data give small features).
template <typename R>
__host__ __device__ inline void gate_features(const Dev &d, int j, const int *st, const int8_t *sx, int S, int I,
                                              float out[24]) {
  int nb[3], xf[3];
  for (int f = 0; f < 3; f++) {
    nb[f] = st[f * S + I];
    xf[f] = sx[f * S + I];
  }
  const R hs = ((const R *)d.hsR)[j];
  const R eps = ((const R *)d.epsA)[j];
  for (int h = 0; h < 2; h++) {
    const int v = h == 0 ? 3 : 0;
    R q[4], g[4][2];
    q[0] = ((const R *)d.dq)[v * d.cs + j];
    img_dg<R>(d, v, j, 0, g[0]);
    for (int f = 0; f < 3; f++) {
      q[1 + f] = img_dq<R>(d, v, nb[f], xf[f]);
      img_dg<R>(d, v, nb[f], xf[f], g[1 + f]);
    }
    R mean = (q[0] + q[1] + q[2] + q[3]) * (R)0.25;
    R raw[12], ss = 0;
    for (int m = 0; m < 4; m++) {
      raw[3 * m] = q[m] - mean;
      raw[3 * m + 1] = hs * g[m][0];
      raw[3 * m + 2] = hs * g[m][1];
    }
    for (int k = 0; k < 12; k++) ss += raw[k] * raw[k];
    R Q0 = q[0] + ((const R *)d.refR)[2 * d.inst[j] + (v == 3 ? 1 : 0)];
    ss += eps * (1 + Q0 * Q0);
    R is = (R)1 / r_sqrt<R>(ss);
    for (int k = 0; k < 12; k++) out[12 * h + k] = (float)(raw[k] * is);
  }
}

#ifdef __CUDACC__
// D = A (16x16 bf16, row) * B (16x8 bf16, col) + D (fp32)
__device__ __forceinline__ void mma_bf16(float d[4], const unsigned a[4], const unsigned b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<unsigned *>(&v);
}
__device__ __forceinline__ unsigned ld_pair(const __nv_bfloat16 *p) { return *reinterpret_cast<const unsigned *>(p); }

// A fragment (16 rows x 16 cols, k offset k0) from a bf16 row-major tile with
// leading dimension ld (elements); lane layout of mma.m16n8k16
__device__ __forceinline__ void load_a(unsigned a[4], const __nv_bfloat16 *t, int ld, int r0, int k0, int lane) {
  const int g = lane >> 2, c = (lane & 3) * 2;
  a[0] = ld_pair(t + (r0 + g) * ld + k0 + c);
  a[1] = ld_pair(t + (r0 + g + 8) * ld + k0 + c);
  a[2] = ld_pair(t + (r0 + g) * ld + k0 + c + 8);
  a[3] = ld_pair(t + (r0 + g + 8) * ld + k0 + c + 8);
}
// B fragment (16 k x 8 n) where element (k, n) = W[n0 + n][k0 + k] of a
// row-major [n][k] bf16 matrix with leading dimension ld
__device__ __forceinline__ void load_b_nk(unsigned b[2], const __nv_bfloat16 *w, int ld, int n0, int k0, int lane) {
  const int g = lane >> 2, c = (lane & 3) * 2;
  b[0] = ld_pair(w + (n0 + g) * ld + k0 + c);
  b[1] = ld_pair(w + (n0 + g) * ld + k0 + c + 8);
}

// Convert the float parameter vector into the tensor-core layout (block-wide),
// for training: the inputs are normalised, then rounded.
__device__ inline void mlp_pack(MlpDev &w, const float *P, float threshold_logit, int tid, int nth) {
  for (int i = tid; i < MLP_H * 32; i += nth) {
    int o = i >> 5, k = i & 31;
    w.w1[i] = __float2bfloat16_rn(k < MLP_IN ? P[MLP_W1 + o * MLP_IN + k] : 0.f);
    w.w2[i] = __float2bfloat16_rn(P[MLP_W2 + o * MLP_H + k]);
  }
  for (int i = tid; i < MLP_H; i += nth) {
    w.b1[i] = P[MLP_B1 + i];
    w.b2[i] = P[MLP_B2 + i];
    w.w3[i] = P[MLP_W3 + i];
  }
  for (int i = tid; i < MLP_IN; i += nth) {
    w.mean[i] = P[MLP_MEAN + i];
    w.istd[i] = P[MLP_ISTD + i];
  }
  if (tid == 0) {
    w.b3 = P[MLP_B3];
    w.threshold = threshold_logit;
  }
}

// The network as B fragments and per-lane bias columns of mma.m16n8k16: a
// warp loads it once and keeps it in registers across many tiles.
struct MlpFrags {
  unsigned w1[2][4][2], w2[2][4][2];   // [k step][n tile][reg]
  float b1[4][2], b2[4][2], w3[4][2];  // columns 8 nt + c, 8 nt + c + 1
  float b3, threshold;
};

__device__ inline void mlp_frags(MlpFrags &F, const MlpDev &w, int lane) {
  const int c = (lane & 3) * 2;
  for (int ks = 0; ks < 2; ks++)
    for (int nt = 0; nt < 4; nt++) {
      load_b_nk(F.w1[ks][nt], w.w1, 32, 8 * nt, 16 * ks, lane);
      load_b_nk(F.w2[ks][nt], w.w2, 32, 8 * nt, 16 * ks, lane);
    }
  for (int nt = 0; nt < 4; nt++)
    for (int i = 0; i < 2; i++) {
      F.b1[nt][i] = w.b1[8 * nt + c + i];
      F.b2[nt][i] = w.b2[8 * nt + c + i];
      F.w3[nt][i] = w.w3[8 * nt + c + i];
    }
  F.b3 = w.b3;
  F.threshold = w.threshold;
}

// The inference image: the input normalisation folded into the first layer,
// W1' = W1 diag(inv_std) (rounded to bf16), b1' = b1 - W1' mean (FP32, in
// input order), so the raw features are rounded and fed in (mean = 0,
// inv_std = 1 in the image).
__device__ inline void mlp_pack_folded(MlpDev &w, const float *P, float threshold_logit, int tid, int nth) {
  for (int i = tid; i < MLP_H * 32; i += nth) {
    int o = i >> 5, k = i & 31;
    w.w1[i] = __float2bfloat16_rn(k < MLP_IN ? P[MLP_W1 + o * MLP_IN + k] * P[MLP_ISTD + k] : 0.f);
    w.w2[i] = __float2bfloat16_rn(P[MLP_W2 + o * MLP_H + k]);
  }
  for (int i = tid; i < MLP_H; i += nth) {
    float b = P[MLP_B1 + i];
    for (int k = 0; k < MLP_IN; k++) b -= P[MLP_W1 + i * MLP_IN + k] * P[MLP_ISTD + k] * P[MLP_MEAN + k];
    w.b1[i] = b;
    w.b2[i] = P[MLP_B2 + i];
    w.w3[i] = P[MLP_W3 + i];
  }
  for (int i = tid; i < MLP_IN; i += nth) {
    w.mean[i] = 0.f;
    w.istd[i] = 1.f;
  }
  if (tid == 0) {
    w.b3 = P[MLP_B3];
    w.threshold = threshold_logit;
  }
}

// One warp: logits of the 16 cells in rows 16 mt .. 16 mt + 15 of X (bf16,
// row stride ld, cols 24..31 zero); lane r < 16 returns the logit of row
// 16 mt + r.
__device__ __forceinline__ void frag_w1(const MlpFrags &F, int ks, int nt, int, unsigned b[2]) {
  b[0] = F.w1[ks][nt][0]; b[1] = F.w1[ks][nt][1];
}
__device__ __forceinline__ void frag_w2(const MlpFrags &F, int ks, int nt, int, unsigned b[2]) {
  b[0] = F.w2[ks][nt][0]; b[1] = F.w2[ks][nt][1];
}
__device__ __forceinline__ float2 frag_b1(const MlpFrags &F, int nt, int) { return make_float2(F.b1[nt][0], F.b1[nt][1]); }
__device__ __forceinline__ float2 frag_b2(const MlpFrags &F, int nt, int) { return make_float2(F.b2[nt][0], F.b2[nt][1]); }
__device__ __forceinline__ float2 frag_w3(const MlpFrags &F, int nt, int) { return make_float2(F.w3[nt][0], F.w3[nt][1]); }
__device__ __forceinline__ float frag_b3(const MlpFrags &F) { return F.b3; }

template <typename Frags>
__device__ inline float mlp_rows16(const Frags &F, const __nv_bfloat16 *X, int ld, int mt, int lane) {
  // layer 1: Z1 = X W1^T, N = 32 (4 tiles), K = 32 (2 steps)
  float z1[4][4];
  for (int nt = 0; nt < 4; nt++)
    for (int i = 0; i < 4; i++) z1[nt][i] = 0.f;
  for (int ks = 0; ks < 2; ks++) {
    unsigned a[4];
    load_a(a, X, ld, 16 * mt, 16 * ks, lane);
    for (int nt = 0; nt < 4; nt++) {
      unsigned b[2];
      frag_w1(F, ks, nt, lane, b);
      mma_bf16(z1[nt], a, b);
    }
  }
  // bias + ReLU, reused in registers as the A operand of layer 2
  unsigned a2[2][4];
  for (int nt = 0; nt < 4; nt++) {
    const float2 bb = frag_b1(F, nt, lane);
    float h0 = fmaxf(z1[nt][0] + bb.x, 0.f), h1 = fmaxf(z1[nt][1] + bb.y, 0.f);
    float h2 = fmaxf(z1[nt][2] + bb.x, 0.f), h3 = fmaxf(z1[nt][3] + bb.y, 0.f);
    int ks = nt >> 1, half = nt & 1;
    a2[ks][2 * half] = pack_bf16(h0, h1);
    a2[ks][2 * half + 1] = pack_bf16(h2, h3);
  }
  float z2[4][4];
  for (int nt = 0; nt < 4; nt++)
    for (int i = 0; i < 4; i++) z2[nt][i] = 0.f;
  for (int ks = 0; ks < 2; ks++)
    for (int nt = 0; nt < 4; nt++) {
      unsigned b[2];
      frag_w2(F, ks, nt, lane, b);
      mma_bf16(z2[nt], a2[ks], b);
    }
  // layer 3 (N = 1) on the FP32 pipes: row g and row g + 8 partial dots
  float s0 = 0.f, s1 = 0.f;
  for (int nt = 0; nt < 4; nt++) {
    const float2 bb = frag_b2(F, nt, lane), ww = frag_w3(F, nt, lane);
    float h0 = fmaxf(z2[nt][0] + bb.x, 0.f), h1 = fmaxf(z2[nt][1] + bb.y, 0.f);
    float h2 = fmaxf(z2[nt][2] + bb.x, 0.f), h3 = fmaxf(z2[nt][3] + bb.y, 0.f);
    // activations are rounded to bf16 like the operands of the tensor-core layers
    h0 = __bfloat162float(__float2bfloat16_rn(h0)); h1 = __bfloat162float(__float2bfloat16_rn(h1));
    h2 = __bfloat162float(__float2bfloat16_rn(h2)); h3 = __bfloat162float(__float2bfloat16_rn(h3));
    s0 += h0 * ww.x + h1 * ww.y;
    s1 += h2 * ww.x + h3 * ww.y;
  }
  s0 += __shfl_xor_sync(0xffffffffu, s0, 1);
  s0 += __shfl_xor_sync(0xffffffffu, s0, 2);
  s1 += __shfl_xor_sync(0xffffffffu, s1, 1);
  s1 += __shfl_xor_sync(0xffffffffu, s1, 2);
  // rows g (s0) and g + 8 (s1) live on lanes 4g..4g+3
  const int src = (lane & 7) * 4;
  const float v0 = __shfl_sync(0xffffffffu, s0, src), v1 = __shfl_sync(0xffffffffu, s1, src);
  return (lane < 8 ? v0 : v1) + frag_b3(F);
}

// One warp: logits of 32 cells; lane r returns the logit of row r.
template <typename Frags>
__device__ inline float mlp_tile32(const Frags &F, const __nv_bfloat16 *X, int ld, int lane) {
  float lo = mlp_rows16(F, X, ld, 0, lane), hi = mlp_rows16(F, X, ld, 1, lane);
  float hi_r = __shfl_sync(0xffffffffu, hi, lane & 15);
  return lane < 16 ? lo : hi_r;
}
#endif

}  // namespace gks2l
