// gks2l: CUDA kernels (sm_103a) and the C ABI of include/gks2l.h.
//
// One S2O4 stage (arXiv 2306.04467, Eq. SWE-fully-discrete) over
// structure-of-arrays data in a Morton-renumbered cell order:
//   k_recon   (32 cells x 6 variables per block) compact P3/WENO reconstruction
//             (Sec. 3.4); the tile's operator rows arrive in shared memory by
//             bulk copy (cp.async.bulk) behind an mbarrier
//   k_iface   (edge x layer)         blended interface levels h-hat (Sec. 2.3)
//   k_edge    (edge x layer x point) gas-kinetic interface solution (Eq. SWE-2nd-order)
//   k_update  (cell)                 fluxes, sources, S2O4 update, Gauss-theorem
//                                    gradients (Eqs. SWE-semi-flux, slope-1, S2O3),
//                                    CFL reduction
// With the learned troubled-cell gate, k_gate (next stage's mask) runs on a
// second stream, and k_iface + k_edge become k_edgef (both in one pass where
// the plane gradients carry no weight) + k_edge_deferred (the other edges).
// A step is k_step_begin + two stages, captured once into a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "gks2l.h"
#include "mlp.cuh"
#include "prep.h"
#include "stage.cuh"
#include "tcgen05.cuh"

using namespace gks2l;

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr unsigned long long DBL_INF_BITS = 0x7FF0000000000000ull;
constexpr int TW = 32;                  // cells per reconstruction tile
constexpr int REF_CHUNK = 4096;         // cells per chunk of the reference-level reduction
constexpr int ST_TIMEOUT = 4;           // status bit: a bounded wait gave up
constexpr int ST_COPY_LOST = 8;         // status bit: the second wait gave up too (copies in flight)
constexpr int GATE_LD = 40;             // padded row stride of the gate feature tile (bank spread)

// ---------------------------------------------------------------- TMA staging
// The reconstruction's operator rows of one tile of TW cells, [row][TW] per
// group, stored contiguously per tile in global memory and copied as they lie
// into shared memory by the bulk-copy engine. The groups come in the order
// the copies need them: what every tile uses (P3 least-squares rows, monomial
// means, stencil cells and their transforms), then what only tiles with a
// troubled cell use (P1 candidate rows, smoothness forms), so a tile the gate
// calls smooth fetches one prefix.
template <typename R> struct TileLayout {
  static constexpr unsigned LSQ = 0;
  static constexpr unsigned MM = LSQ + kCoef * kCols * TW * sizeof(R);
  static constexpr unsigned ST = MM + 7 * TW * sizeof(R);
  static constexpr unsigned SX = ST + kSlots * TW * 4;
  static constexpr unsigned P1 = SX + kSlots * TW;
  static constexpr unsigned BQ = P1 + 30 * TW * sizeof(R);
  static constexpr unsigned END = BQ + kBeta * TW * sizeof(R);
  static constexpr unsigned TILE = (END + 127) / 128 * 128;   // tile stride in global memory
  static constexpr unsigned TX_LINEAR = P1;                    // bytes of the first copy
  static constexpr unsigned TX2 = END - P1;                    // bytes of the second copy
  // Shared memory holds the first copy; a tile with a troubled cell fetches
  // the second after the P3 fit, into the space of the LSQ rows, which the
  // side-record staging then follows.
  static constexpr unsigned LATE = LSQ;
  static constexpr unsigned STG = LATE + (TX2 + 127) / 128 * 128;
  static constexpr unsigned BAR = (P1 + 127) / 128 * 128;      // the mbarrier, after the first copy
  static_assert(STG + 2 * TW * NREC * sizeof(R) <= MM, "late rows and side-record staging fit in the LSQ rows");
  static_assert(P1 % 16 == 0 && END % 16 == 0, "bulk copies move multiples of 16 bytes");
};

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned)
// from global to shared memory, completing on the mbarrier
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, void *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"((unsigned long long)__cvta_generic_to_global(src)), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(void *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// wait for the phase of the given parity of an mbarrier for at most ~limit_ns
// and at most max_polls polls
__device__ __forceinline__ bool mbar_wait_bounded(void *bar, unsigned parity, unsigned long long limit_ns,
                                                  int max_polls = 1 << 24) {
  unsigned long long t0 = global_ns();
  for (int it = 0; it < max_polls; it++) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
  return false;
}

// ------------------------------------------------------------------ kernels
// resident reconstruction blocks per SM the register budget is held to (in
// FP32 eight, as many as the registers allow: a block per tile keeps 48
// warps per SM on the neighbour gathers; persistent blocks with two operator
// buffers, fetching the next tile during the current one, halve the warps
// and run slower)
template <typename R> struct ReconOcc { static constexpr int value = 8; };
template <> struct ReconOcc<double> { static constexpr int value = 4; };
template <typename R> constexpr unsigned recon_smem() { return TileLayout<R>::BAR + 16; }

// Positivity option (not in the paper), on a tile's staged side records: for
// each cell and layer the least depth at the cell's six edge Gauss points;
// below pos_floor times the cell-average depth, the layer's depth and
// discharge polynomials are scaled toward their averages by one factor so
// that it meets the floor (the lower layer's level keeps the bottom's linear
// part); a layer whose point depths dip below half its average is flagged
// for the edge solution's velocity bound. One thread per (cell, layer).
template <typename R>
__device__ void recon_positivity(const Dev &d, const Par &p, int j, int lay, R *rec) {
  const int N = d.cs, NE = d.ne;
  const R *xl = (const R *)d.exiL, *xr = (const R *)d.exiR;
  R hmin = (R)INFINITY;
  for (int f = 0; f < 3; f++) {
    const int ce = d.cedge[f * N + j], e = ce >= 0 ? ce : ~ce;
    const R *xs = ce >= 0 ? xl : xr;
    for (int q = 0; q < 2; q++) {
      const R x = xs[(2 * q) * NE + e], y = xs[(2 * q + 1) * NE + e];
      R v[3];
      rec_values<R>(rec, x, y, v);
      const R h = ref_depth<R>(d, lay, e, q) + v[0];
      hmin = h < hmin ? h : hmin;
    }
  }
  const R hbar = lay == 0 ? ((const R *)d.hrefc)[j] + rec[10] : ((const R *)d.refR)[2 * d.inst[j]] + rec[10];
  ((R *)d.pos_hbar)[lay * N + j] = hbar;
  d.pos_flag[lay * N + j] = hmin < (R)0.5 * hbar ? 1 : 0;
  const R fl = (R)p.pos_floor * hbar;
  if (!(hmin < fl)) return;
  R th = (hbar - fl) / (hbar - hmin);
  th = th > (R)0 ? th : (R)0;
  for (int i = 0; i < 3; i++)
    for (int k = 0; k < 10; k++) rec[12 * i + k] *= th;
  if (lay == 0) {
    // eta1 = h1 + B: the bottom's linear part (slope x cell scale) stays
    const R ih = rec[11];
    rec[1] += ((R)1 - th) * rec[23] / ih;
    rec[2] += ((R)1 - th) * rec[35] / ih;
  }
}

template <typename R, bool POS = false>
__global__ void __launch_bounds__(192, ReconOcc<R>::value) k_recon(Dev d, Par p) {
  using T = TileLayout<R>;
  extern __shared__ __align__(128) unsigned char sm[];
  const int j0 = blockIdx.x * TW;
  void *bar = sm + T::BAR;
  // troubled-cell gate: the previous reconstruction left the mask of this
  // tile's cells it calls smooth; a tile whose cells all take the linear
  // weights needs neither the P1 rows nor the smoothness forms
  const bool gate_on = p.use_gate && !p.harvest;
  const unsigned lin_mask = gate_on ? d.gate_mask[blockIdx.x] : 0u;
  const bool all_linear = lin_mask == 0xffffffffu;
  const bool lead = threadIdx.x == 0 && threadIdx.y == 0;
  const unsigned char *src = (const unsigned char *)d.ops + (size_t)blockIdx.x * T::TILE;
  if (lead) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(T::TX_LINEAR)
                 : "memory");
    bulk_load(sm, src, T::TX_LINEAR, bar);
  }
  // the cell's activity (a chain of two loads) resolves during the copies
  const int j = j0 + threadIdx.x, v = threadIdx.y;
  const bool active = j < d.nt && (p.all_active || d.dt[d.inst[j]] > 0);
  __syncthreads();
  const bool landed =
      mbar_wait_bounded(bar, 0, 1000000000ull, p.staging_polls > 0 ? p.staging_polls - 1 : (1 << 24));
  if (!__syncthreads_and(landed)) {
    // the copies did not land in time: report, wait for them once more
    // (bounded, a second) so no copy outlives the block, and leave (all
    // threads); if they still have not landed, the block's shared memory may
    // yet be written after it exits, which a second bit records
    if (lead) atomicOr(d.status, ST_TIMEOUT);
    if (!landed && !mbar_wait_bounded(bar, 0, 1000000000ull)) atomicOr(d.status, ST_COPY_LOST);
    return;
  }
  CellOps<R> o;
  o.lsq = (const R *)(sm + T::LSQ);
  o.p1 = (const R *)(sm + T::LATE);
  o.bq = (const R *)(sm + T::LATE + (T::BQ - T::P1));
  o.mm = (const R *)(sm + T::MM);
  o.st = (const int *)(sm + T::ST);
  o.sx = (const int8_t *)(sm + T::SX);
  o.stride = TW;
  o.idx = threadIdx.x;
  const bool linear = ((lin_mask >> threadIdx.x) & 1u) != 0;
  if (gate_on && v == 0) {
    const unsigned ns = __popc(__ballot_sync(FULL, active && linear)), nc = __popc(__ballot_sync(FULL, active));
    if (threadIdx.x == 0) {
      atomicAdd(&d.gate_count[0], (unsigned long long)ns);
      atomicAdd(&d.gate_count[1], (unsigned long long)nc);
    }
  }
  R rhs[NCOL], a[9];
  if (active) {
    recon_gather<R>(d, o, j, v, rhs);
    recon_p3<R>(o, rhs, a);
  }
  // every warp is done with the LSQ rows: their space takes the late rows
  // (tiles with a troubled cell) and stages the side records
  __syncthreads();
  if (!all_linear) {
    if (lead) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(T::TX2)
                   : "memory");
      bulk_load(sm + T::LATE, src + T::P1, T::TX2, bar);
    }
    const bool late = mbar_wait_bounded(bar, 1, 1000000000ull);
    if (!__syncthreads_and(late)) {
      if (lead) atomicOr(d.status, ST_TIMEOUT);
      if (!late && !mbar_wait_bounded(bar, 1, 1000000000ull)) atomicOr(d.status, ST_COPY_LOST);
      return;
    }
  }
  R *stg = (R *)(sm + T::STG);
  if (active) recon_finish<R>(d, p, o, j, v, rhs, a, linear, stg);
  if (v == 5 && j < d.nt) {
    // the constant words: 1/h_s and the bottom slope
    R *r0 = stg + (size_t)threadIdx.x * NREC, *r1 = stg + (size_t)(TW + threadIdx.x) * NREC;
    const R ih = ((const R *)d.ihsR)[j];
    r0[11] = ih;
    r1[11] = ih;
    r0[23] = ((const R *)d.bgR)[j];
    r0[35] = ((const R *)d.bgR)[d.cs + j];
    r1[23] = r1[35] = 0;
  }
  __syncthreads();
  if (POS) {
    if (threadIdx.y < 2 && j < d.nt && active) {
      recon_positivity<R>(d, p, j, threadIdx.y, stg + ((size_t)threadIdx.y * TW + threadIdx.x) * NREC);
    }
    __syncthreads();
  }
  // coalesced write-out: each layer's records of the tile are contiguous, and
  // so is the staging tile, so the copy moves 16-byte vectors
  constexpr int V = 16 / sizeof(R);                 // values per vector
  constexpr int NV_LAYER = TW * NREC / V;           // vectors per layer
  const int tid = threadIdx.y * TW + threadIdx.x;
  const int ncell = min(TW, d.nt - j0);             // the last tile may be partial
  for (int i = tid; i < 2 * NV_LAYER; i += TW * 6) {
    const int lay = i / NV_LAYER, r = i - lay * NV_LAYER;
    if (r * V < ncell * NREC)
      reinterpret_cast<uint4 *>((R *)d.srec + ((size_t)lay * d.cs + j0) * NREC)[r] =
          reinterpret_cast<const uint4 *>(stg + lay * TW * NREC)[r];
  }
}

// Troubled-cell gate (not part of the paper). It runs on a second stream
// beside the interface and edge kernels of a stage, on the state that stage
// reconstructed, and leaves for the next reconstruction the mask of cells it
// calls smooth. Persistent warps keep the network in registers and walk over
// tiles of 32 cells: the 24 features of each cell go to a shared-memory tile,
// the network runs on the tensor cores, and the warp writes the tile's mask
// (cells past the end or of finished instances count as smooth).
constexpr int GATE_BLOCKS_PER_SM = 2;

template <typename R>
__global__ void __launch_bounds__(128) k_gate(Dev d, Par p) {
  __shared__ __align__(16) __nv_bfloat16 Xs[4][32 * GATE_LD];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const MlpDev &w = *reinterpret_cast<const MlpDev *>(d.mlp);
  MlpFrags F;
  mlp_frags(F, w, lane);
  __nv_bfloat16 *X = Xs[wid];
  unsigned *row = reinterpret_cast<unsigned *>(X + lane * GATE_LD);
  for (int k = 12; k < 16; k++) row[k] = 0u;   // columns 24..31 stay zero
  const int ntile = (d.nt + TW - 1) / TW;
  for (int tile = blockIdx.x * 4 + wid; tile < ntile; tile += gridDim.x * 4) {
    const int j = tile * TW + lane;
    const bool active = j < d.nt && (p.all_active || d.dt[d.inst[j]] > 0);
    float f[24];
    if (active) {
      gate_features<R>(d, j, d.st_cell, d.st_xf, d.cs, j, f);
    } else {
      for (int k = 0; k < 24; k++) f[k] = 0.f;
    }
    // the image has the input normalisation folded into the first layer
    for (int k = 0; k < 12; k++) row[k] = pack_bf16(f[2 * k], f[2 * k + 1]);
    __syncwarp();
    const float logit = mlp_tile32(F, X, GATE_LD, lane);
    const bool smooth = active && logit < F.threshold;
    const unsigned mask = __ballot_sync(FULL, smooth || !active);
    if (lane == 0) d.gate_next[tile] = mask;
    if (p.logit_out && j < d.nt) p.logit_out[j] = logit;
    __syncwarp();   // the tile is rewritten next
  }
}

// The same gate on the fifth-generation tensor cores: a CTA of 128 threads
// takes 128 cells at a time, one per thread. Each thread writes its cell's
// 24 features (BF16, normalisation folded into the first layer) as one row
// of the A operand in shared memory; one thread issues the layer's MMAs
// (M = 128, N = 32, K = 2 x 16, BF16 in, FP32 out) into tensor memory; each
// warp reads its 32 rows back, adds the bias, applies ReLU and rounds to
// BF16 (the next layer's A operand), and the output layer (N = 1) runs on
// the FP32 pipes. The weights sit in shared memory, not registers. Waits on
// the MMAs' completion are bounded: a wait that gives up records the
// timeout, waits once more and the CTA frees its tensor memory and leaves.
constexpr int GATE_TC_M = 128;
constexpr unsigned GATE_TC_COLS = 32;   // tensor-memory columns: the 32 FP32 outputs of a layer
struct GateTcSmem {
  alignas(128) unsigned char x[GATE_TC_M * 64];   // [128][32] BF16 features, operand layout
  alignas(128) unsigned char h[GATE_TC_M * 64];   // [128][32] BF16 layer-1 activations
  alignas(128) unsigned char w1[32 * 64];         // [32 out][32 in] BF16
  alignas(128) unsigned char w2[32 * 64];
  float b1[32], b2[32], w3[32];
  float b3, threshold;
  alignas(8) unsigned long long bar;
  uint32_t tmem;
};

__device__ __forceinline__ uint4 pack8_bf16(const float *v) {
  uint4 r;
  r.x = pack_bf16(v[0], v[1]);
  r.y = pack_bf16(v[2], v[3]);
  r.z = pack_bf16(v[4], v[5]);
  r.w = pack_bf16(v[6], v[7]);
  return r;
}

template <typename R>
__global__ void __launch_bounds__(GATE_TC_M) k_gate_tc(Dev d, Par p) {
  __shared__ GateTcSmem S;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const MlpDev &w = *reinterpret_cast<const MlpDev *>(d.mlp);
  for (int i = tid; i < 32 * 32; i += GATE_TC_M) {
    const int n = i >> 5, k = i & 31;
    *reinterpret_cast<__nv_bfloat16 *>(S.w1 + tc::tile_offset(n, k)) = w.w1[i];
    *reinterpret_cast<__nv_bfloat16 *>(S.w2 + tc::tile_offset(n, k)) = w.w2[i];
  }
  if (tid < 32) {
    S.b1[tid] = w.b1[tid];
    S.b2[tid] = w.b2[tid];
    S.w3[tid] = w.w3[tid];
  }
  if (tid == 0) {
    S.b3 = w.b3;
    S.threshold = w.threshold;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&S.bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tc::alloc(&S.tmem, GATE_TC_COLS);
  tc::fence_proxy();        // the weight tiles, for the tensor cores
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = S.tmem, twarp = tbase + ((uint32_t)(warp * 32) << 16);
  const uint32_t idesc = tc::idesc_bf16(GATE_TC_M, 32);
  const unsigned ax = smem_addr(S.x), ah = smem_addr(S.h), a1 = smem_addr(S.w1), a2 = smem_addr(S.w2);
  const int ntile = (d.nt + GATE_TC_M - 1) / GATE_TC_M, nword = (d.nt + TW - 1) / TW;
  unsigned phase = 0;
  bool failed = false;
  for (int tile = blockIdx.x; tile < ntile && !failed; tile += gridDim.x) {
    const int j = tile * GATE_TC_M + tid;
    const bool active = j < d.nt && (p.all_active || d.dt[d.inst[j]] > 0);
    float f[32];
    if (active) gate_features<R>(d, j, d.st_cell, d.st_xf, d.cs, j, f);
    else
      for (int k = 0; k < 24; k++) f[k] = 0.f;
    for (int k = 24; k < 32; k++) f[k] = 0.f;
    for (int c = 0; c < 4; c++) *reinterpret_cast<uint4 *>(S.x + tc::tile_offset(tid, 8 * c)) = pack8_bf16(f + 8 * c);
    float z[32], logit = 0.f;
    for (int layer = 0; layer < 2 && !failed; layer++) {
      tc::fence_proxy();
      tc::fence_before();
      __syncthreads();
      if (tid == 0) {
        tc::fence_after();
        const unsigned a = layer == 0 ? ax : ah, b = layer == 0 ? a1 : a2;
        tc::mma_bf16(tbase, tc::smem_desc(a), tc::smem_desc(b), idesc, 0);
        tc::mma_bf16(tbase, tc::smem_desc(a + 2 * tc::kLbo), tc::smem_desc(b + 2 * tc::kLbo), idesc, 1);
        tc::commit(&S.bar);
      }
      const bool done = mbar_wait_bounded(&S.bar, phase, 1000000000ull);
      if (!__syncthreads_and(done)) {
        // record, wait once more so no MMA outlives the tensor memory, leave
        if (tid == 0) atomicOr(d.status, ST_TIMEOUT);
        if (!done && !mbar_wait_bounded(&S.bar, phase, 1000000000ull)) atomicOr(d.status, ST_COPY_LOST);
        failed = true;
        break;
      }
      phase ^= 1u;
      tc::fence_after();
      tc::ld32(twarp, z);
      if (layer == 0) {
        for (int k = 0; k < 32; k++) z[k] = fmaxf(z[k] + S.b1[k], 0.f);
        for (int c = 0; c < 4; c++)
          *reinterpret_cast<uint4 *>(S.h + tc::tile_offset(tid, 8 * c)) = pack8_bf16(z + 8 * c);
      } else {
        // activations rounded to BF16 like the operands of the tensor-core layers
        float s0 = 0.f, s1 = 0.f;
        for (int k = 0; k < 32; k += 2) {
          s0 += __bfloat162float(__float2bfloat16_rn(fmaxf(z[k] + S.b2[k], 0.f))) * S.w3[k];
          s1 += __bfloat162float(__float2bfloat16_rn(fmaxf(z[k + 1] + S.b2[k + 1], 0.f))) * S.w3[k + 1];
        }
        logit = s0 + s1 + S.b3;
      }
    }
    if (failed) break;
    const bool smooth = active && logit < S.threshold;
    const unsigned mask = __ballot_sync(FULL, smooth || !active);
    const int word = tile * (GATE_TC_M / TW) + warp;
    if (lane == 0 && word < nword) d.gate_next[word] = mask;
    if (p.logit_out && j < d.nt) p.logit_out[j] = logit;
    tc::fence_before();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 0) tc::dealloc(tbase, GATE_TC_COLS);
}

// gate network image for the reconstruction blocks (one block)
__global__ void k_mlp_pack(const float *P, float threshold_logit, MlpDev *out) {
  mlp_pack_folded(*out, P, threshold_logit, threadIdx.x, blockDim.x);
}

// training data for the gate, written in the caller's cell order: 24
// features, the label (largest departure of the WENO weights from the linear
// ones over the six variables above tol) and, if asked, the gate logits the
// reconstruction computed
template <typename R>
__global__ void k_harvest(Dev d, const int *perm, float tol, const float *logit_dev, float *X, float *y,
                          float *logits) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= d.nt) return;
  const size_t c = (size_t)perm[j];
  float f[24];
  gate_features<R>(d, j, d.st_cell, d.st_xf, d.cs, j, f);
  for (int k = 0; k < 24; k++) X[c * 24 + k] = f[k];
  float dv = 0.f;
  for (int v = 0; v < NV; v++) dv = fmaxf(dv, d.wdev[v * d.cs + j]);
  y[c] = dv > tol ? 1.f : 0.f;
  if (logits) logits[c] = logit_dev[j];
}

// Each side's own level of layer ell, the mean over the edge's two points:
// the q = 0 thread writes the L side's, the q = 1 thread the R side's.
template <typename R>
__device__ __forceinline__ void own_write(const Dev &d, int e, int ell, int q, const R own[2], bool ok) {
  const R mine = q == 0 ? own[0] : own[1], theirs = q == 0 ? own[1] : own[0];
  const R m = (R)0.5 * (mine + __shfl_xor_sync(FULL, theirs, 1));
  if (ok) ((R *)d.eO)[(2 * q + ell) * d.ne + e] = m;
}

// An edge's results for layer ell: the Gauss point q = 0 thread holds the
// averaged F and F_t, the q = 1 thread W and W_t (avg[0..2], avg[3..5]). The
// depth components of F and F_t also go out in FP64 for the cells' mass sums.
// Stage 2 keeps only W_t: the stage-end interface values take the stage-1
// W^n(x) (Eq. S2O3) and the interlayer source the cells' own levels.
template <typename R>
__device__ __forceinline__ void edge_write(const Dev &d, int e, int ell, int q, int stage, const R avg[6]) {
  const int NE = d.ne;
  const int vb = ell == 0 ? 3 : 0;
  R *A = (R *)(q == 0 ? d.eF : d.eWn);
  R *B = (R *)(q == 0 ? d.eFt : d.eWt);
  const bool wa = q == 0 || stage == 1;
  for (int k = 0; k < 3; k++) {
    if (wa) A[(vb + k) * NE + e] = avg[k];
    B[(vb + k) * NE + e] = avg[3 + k];
  }
  if (q == 0) {
    d.eFm[(vb / 3) * NE + e] = (double)avg[0];
    d.eFtm[(vb / 3) * NE + e] = (double)avg[3];
  }
}

template <typename R>
__device__ __forceinline__ void iface_body(const Dev &d) {
  int tid = blockIdx.x * blockDim.x + threadIdx.x;
  int e = tid >> 1, ell = tid & 1;
  if (e >= d.ne || !(d.dt[d.inst[d.eL[e]]] > 0)) return;
  ((R *)d.hc)[ell * d.ne + e] = iface_unit<R>(d, e, ell);
}

template <typename R, bool POS = false>
__device__ __forceinline__ void edge_body(const Dev &d, const Par &p, int stage) {
  int tid = blockIdx.x * blockDim.x + threadIdx.x;
  int e = tid >> 2, ell = (tid >> 1) & 1, q = tid & 1;
  const int ee = e < d.ne ? e : d.ne - 1;
  // every thread computes (past the last edge: the last edge again), before
  // its instance's dt is known, so the unit's loads issue at once; only
  // edges of instances still running are written
  R out[12], own[2];
  edge_unit<R, false, true, POS>(d, p, ee, ell, q, stage, out, nullptr, own);
  const bool ok = e < d.ne && d.dt[d.inst[d.eL[ee]]] > 0;
  own_write<R>(d, e, ell, q, own, ok);
  // the Gauss point q = 0 thread averages the fluxes (out[0..5]), the q = 1
  // thread the interface values (out[6..11]): each sends the other its half
  R avg[6];
#pragma unroll
  for (int k = 0; k < 6; k++) {
    const R mine = q == 0 ? out[k] : out[6 + k], theirs = q == 0 ? out[6 + k] : out[k];
    avg[k] = (R)0.5 * (mine + __shfl_xor_sync(FULL, theirs, 1));
  }
  if (!ok) return;
  edge_write<R>(d, e, ell, q, stage, avg);
}

// Gated runs: the interface levels and the edge solution in one kernel. Each
// (edge, layer, point) thread evaluates both sides once, forms the point's
// blended level (the pair's mean is the edge's, written to hc) and, where the
// blend weight is 1, the solution; the other (edge, layer) units go to the
// worklist for k_edge_deferred, which runs once every blended level exists.
template <typename R>
__device__ __forceinline__ void edge_fused_body(const Dev &d, const Par &p, int stage) {
  int tid = blockIdx.x * blockDim.x + threadIdx.x;
  int e = tid >> 2, ell = (tid >> 1) & 1, q = tid & 1;
  const int ee = e < d.ne ? e : d.ne - 1;
  R out[12], bl = 0, own[2];
  const bool done = edge_unit<R, true, true>(d, p, ee, ell, q, stage, out, &bl, own);
  if (!done) {
    for (int k = 0; k < 12; k++) out[k] = 0;
  }
  // the edge's blended level: the mean over its two points, summed in point
  // order as the interface kernel sums it
  const R bo = __shfl_xor_sync(FULL, bl, 1);
  const R hcv = Rn<R>::mul((R)0.5, q == 0 ? Rn<R>::add(bl, bo) : Rn<R>::add(bo, bl));
  R avg[6];
#pragma unroll
  for (int k = 0; k < 6; k++) {
    const R mine = q == 0 ? out[k] : out[6 + k], theirs = q == 0 ? out[6 + k] : out[k];
    avg[k] = (R)0.5 * (mine + __shfl_xor_sync(FULL, theirs, 1));
  }
  const bool ok = e < d.ne && d.dt[d.inst[d.eL[ee]]] > 0;
  own_write<R>(d, e, ell, q, own, ok);
  // deferred units to the worklist, one atomic per warp
  const bool push = ok && q == 0 && !done;
  const unsigned bal = __ballot_sync(FULL, push);
  if (bal) {
    const int lane = threadIdx.x & 31, leader = __ffs(bal) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(d.wl_count, __popc(bal));
    base = __shfl_sync(FULL, base, leader);
    if (push) d.wl[base + __popc(bal & ((1u << lane) - 1u))] = (e << 1) | ell;
  }
  if (!ok) return;
  const int NE = d.ne;
  if (q == 0) ((R *)d.hc)[ell * NE + e] = hcv;
  if (!done) return;
  edge_write<R>(d, e, ell, q, stage, avg);
}

// The worklist's units with the plane gradients (every blended level is
// written by now): warps walk it 16 units at a time, a thread pair per unit.
constexpr int DEFER_BLOCKS_PER_SM = 4;

template <typename R>
__global__ void __launch_bounds__(128) k_edge_deferred(Dev d, Par p, int stage) {
  const int n = *d.wl_count;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarp = (gridDim.x * blockDim.x) >> 5;
  for (int base = warp * 16; base < n; base += nwarp * 16) {
    const int i = base + (lane >> 1), q = lane & 1;
    const int item = d.wl[i < n ? i : n - 1];
    const int e = item >> 1, ell = item & 1;
    R out[12];
    edge_unit<R>(d, p, e, ell, q, stage, out);
    R avg[6];
#pragma unroll
    for (int k = 0; k < 6; k++) {
      const R mine = q == 0 ? out[k] : out[6 + k], theirs = q == 0 ? out[6 + k] : out[k];
      avg[k] = (R)0.5 * (mine + __shfl_xor_sync(FULL, theirs, 1));
    }
    if (i >= n) continue;
    edge_write<R>(d, e, ell, q, stage, avg);
  }
}

// min over the warp of non-negative doubles (or +inf): their bit patterns
// order like the values, so the comparison runs on the integer pipes
__device__ __forceinline__ double warp_min(double v) {
  unsigned long long b = (unsigned long long)__double_as_longlong(v);
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long u = __shfl_xor_sync(FULL, b, o);
    b = u < b ? u : b;
  }
  return __longlong_as_double((long long)b);
}
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

// min of dX/U_max per instance, reduced per warp when the warp lies in one
// instance (the usual case), per lane otherwise
__device__ __forceinline__ void reduce_cfl(const Dev &d, bool ok, int inst, double ratio) {
  int lane = threadIdx.x & 31;
  int i0 = __shfl_sync(FULL, inst, 0);
  bool uniform = __all_sync(FULL, !ok || inst == i0) && __shfl_sync(FULL, ok ? 1 : 0, 0);
  if (uniform) {
    double r = warp_min(ok ? ratio : INFINITY);
    if (lane == 0 && r < INFINITY) atomicMin(&d.dtbits[i0], (unsigned long long)__double_as_longlong(r));
  } else if (ok && ratio < INFINITY) {
    atomicMin(&d.dtbits[inst], (unsigned long long)__double_as_longlong(ratio));
  }
}

// per-layer masses of the current state, per instance (FP64 sums; taken when
// the statistics are read, not in the stage kernels)
__global__ void k_mass(Dev d) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  bool ok = j < d.nt;
  int inst = ok ? d.inst[j] : 0;
  double m1 = ok ? d.area[j] * d.avg[3 * d.cs + j] : 0.0, m2 = ok ? d.area[j] * d.avg[j] : 0.0;
  int lane = threadIdx.x & 31;
  int i0 = __shfl_sync(FULL, inst, 0);
  bool uniform = __all_sync(FULL, !ok || inst == i0) && __shfl_sync(FULL, ok ? 1 : 0, 0);
  if (uniform) {
    double s1 = warp_sum(m1), s2 = warp_sum(m2);
    if (lane == 0) {
      atomicAdd(&d.mass[2 * i0], s1);
      atomicAdd(&d.mass[2 * i0 + 1], s2);
    }
  } else if (ok) {
    atomicAdd(&d.mass[2 * inst], m1);
    atomicAdd(&d.mass[2 * inst + 1], m2);
  }
}

template <typename R>
__device__ __forceinline__ void update_body(const Dev &d, const Par &p, int stage) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  bool ok = j < d.nt;
  int inst = ok ? d.inst[j] : 0;
  double ratio = INFINITY;
  int fl = 0;
  if (ok) {
    double r = update_unit<R>(d, p, j, stage, &fl);
    if (r > 0) ratio = r;
  }
  if (fl) atomicOr(d.status, fl);
  // the gate has joined: its mask becomes the next reconstruction's
  if (p.use_gate && ok && (j & (TW - 1)) == 0) d.gate_mask[j / TW] = d.gate_next[j / TW];
  if (stage != 2) return;
  reduce_cfl(d, ok, inst, ratio);
  if (ok && j == d.inst_first[inst]) d.t[inst] += d.dt[inst];
}

// The interface, edge (fused edge) and update kernels come in five launch
// shapes (threads per block, and for two of them a register budget); the
// autotuner (gks2l_autotune) picks one per kernel. The bodies are shared;
// the entry points differ in their launch bounds only.
template <typename R, int BS>
__global__ void __launch_bounds__(BS) k_iface(Dev d) { iface_body<R>(d); }
template <typename R, int BS>
__global__ void __launch_bounds__(BS) k_edge(Dev d, Par p, int stage) { edge_body<R>(d, p, stage); }
// (the fused kernel's default shapes are held to 768 resident threads per SM,
// the 80 registers its body compiles to when left alone)
template <typename R, int BS>
__global__ void __launch_bounds__(BS, 768 / BS) k_edgef(Dev d, Par p, int stage) { edge_fused_body<R>(d, p, stage); }
template <typename R, int BS>
__global__ void __launch_bounds__(BS) k_update(Dev d, Par p, int stage) { update_body<R>(d, p, stage); }
// the edge solution with the positivity option (one launch shape)
template <typename R>
__global__ void __launch_bounds__(128) k_edge_pos(Dev d, Par p, int stage) { edge_body<R, true>(d, p, stage); }
template <typename R>
__global__ void __launch_bounds__(128, 8) k_iface_r64(Dev d) { iface_body<R>(d); }
template <typename R>
__global__ void __launch_bounds__(128, 8) k_edge_r64(Dev d, Par p, int stage) { edge_body<R>(d, p, stage); }
template <typename R>
__global__ void __launch_bounds__(128, 8) k_edgef_r64(Dev d, Par p, int stage) { edge_fused_body<R>(d, p, stage); }
template <typename R>
__global__ void __launch_bounds__(128, 8) k_update_r64(Dev d, Par p, int stage) { update_body<R>(d, p, stage); }
template <typename R>
__global__ void __launch_bounds__(128, 4) k_iface_r128(Dev d) { iface_body<R>(d); }
template <typename R>
__global__ void __launch_bounds__(128, 4) k_edge_r128(Dev d, Par p, int stage) { edge_body<R>(d, p, stage); }
template <typename R>
__global__ void __launch_bounds__(128, 4) k_edgef_r128(Dev d, Par p, int stage) { edge_fused_body<R>(d, p, stage); }
template <typename R>
__global__ void __launch_bounds__(128, 4) k_update_r128(Dev d, Par p, int stage) { update_body<R>(d, p, stage); }

// CFL ratio of the current state (after a state is set), in the form's
// precision as the update kernel computes it; a depth <= 0 or a non-finite
// value is recorded
template <typename R>
__global__ void __launch_bounds__(128) k_cfl(Dev d, Par p) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  bool ok = j < d.nt;
  int inst = ok ? d.inst[j] : 0;
  double ratio = INFINITY;
  if (ok) {
    double w[NV];
    int fl = 0;
    for (int v = 0; v < NV; v++) {
      w[v] = d.avg[v * d.cs + j];
      if (!isfinite(w[v])) fl = 2;
    }
    if (!fl && (w[0] <= 0 || w[3] <= 0)) fl = 1;
    if (!fl) {
      ratio = cfl_ratio<R>(w, d.dX[j], pv<R>(p.g, p.gf));
      if (!(ratio > 0) || !isfinite(ratio)) fl = 2;
    }
    if (fl) {
      atomicOr(d.status, fl);
      ratio = INFINITY;
    }
  }
  reduce_cfl(d, ok, inst, ratio);
}

// Reference levels of each instance (R2, R1): the area-weighted means of h2
// and eta1 = h1 + B, rounded to 2^-32. Deterministic: fixed chunks of an
// instance's cells, each summed in a fixed order (thread-strided, then a
// shared-memory tree), then the chunks in order by one thread per instance.
constexpr int REF_THREADS = 256;
__global__ void __launch_bounds__(REF_THREADS) k_ref_partial(Dev d, const int *chunk, double *part) {
  __shared__ double sh[3][REF_THREADS];
  const int c = blockIdx.x, t = threadIdx.x, j1 = chunk[2 * c + 1];
  double a = 0, s2 = 0, s1 = 0;
  for (int j = chunk[2 * c] + t; j < j1; j += REF_THREADS) {
    const double w = d.area[j];
    a += w;
    s2 += w * d.avg[j];
    s1 += w * (d.avg[3 * d.cs + j] + d.bmean[j]);
  }
  sh[0][t] = a;
  sh[1][t] = s2;
  sh[2][t] = s1;
  __syncthreads();
  for (int o = REF_THREADS / 2; o > 0; o >>= 1) {
    if (t < o)
      for (int k = 0; k < 3; k++) sh[k][t] += sh[k][t + o];
    __syncthreads();
  }
  if (t < 3) part[3 * c + t] = sh[t][0];
}

template <typename R>
__global__ void k_ref_final(Dev d, const int *inst_chunk, const double *part) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.ninst) return;
  double a = 0, s2 = 0, s1 = 0;
  for (int c = inst_chunk[i]; c < inst_chunk[i + 1]; c++) {
    a += part[3 * c];
    s2 += part[3 * c + 1];
    s1 += part[3 * c + 2];
  }
  const double r2 = ldexp(rint(ldexp(s2 / a, 32)), -32), r1 = ldexp(rint(ldexp(s1 / a, 32)), -32);
  d.ref[2 * i] = r2;
  d.ref[2 * i + 1] = r1;
  ((R *)d.refR)[2 * i] = (R)r2;
  ((R *)d.refR)[2 * i + 1] = (R)r1;
}

__global__ void k_reset_stats(Dev d) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.ninst) return;
  d.dtbits[i] = DBL_INF_BITS;
}

// step size of each instance from the CFL ratio of the current state (Sec. 4),
// shortened to land on t_end
template <typename R>
__global__ void k_step_begin(Dev d, Par p, const double *tend) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.ninst) return;
  double r = __longlong_as_double((long long)d.dtbits[i]);
  double dt = p.cfl * r;
  double te = *tend;
  if (te > 0) {
    double rem = te - d.t[i];
    if (rem <= 1e-12 * fmax(1.0, fabs(te))) dt = 0;
    else if (dt > rem) dt = rem;
  }
  if (!isfinite(dt) || dt < 0) {
    atomicOr(d.status, 2);
    dt = 0;
  }
  d.dt[i] = dt;
  ((R *)d.dtR)[i] = (R)dt;
  d.dtbits[i] = DBL_INF_BITS;
}

// deviation mirrors of a freshly set state: dq, dg (gradients given in the
// caller's order, stored as given), R1 - B per cell
template <typename R>
__global__ void k_mirrors(Dev d, const int *perm, const double *grad_caller) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= d.nt) return;
  const int N = d.cs, in = d.inst[j], c = perm[j];
  R *dq = (R *)d.dq, *dg = (R *)d.dg;
  const double R2 = d.ref[2 * in], R1 = d.ref[2 * in + 1];
  dq[j] = (R)(d.avg[j] - R2);
  dq[3 * N + j] = (R)((d.avg[3 * N + j] + d.bmean[j]) - R1);
  for (int v : {1, 2, 4, 5}) dq[v * N + j] = (R)d.avg[v * N + j];
  for (int k = 0; k < 12; k++) dg[k * N + j] = (R)(grad_caller ? grad_caller[(size_t)k * d.nt + c] : 0.0);
  ((R *)d.hrefc)[j] = (R)(R1 - d.bmean[j]);
}

template <typename R>
__global__ void k_edge_ref(Dev d) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.ne) return;
  const double R1 = d.ref[2 * d.inst[d.eL[e]] + 1];
  ((R *)d.hrefe)[e] = (R)(R1 - d.eb0[e]);
  ((R *)d.hrefe)[d.ne + e] = (R)(R1 - d.eb1[e]);
}

// gradients in the caller's order
template <typename R>
__global__ void k_grad_out(Dev d, const int *perm, double *out) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= d.nt) return;
  const int c = perm[j];
  const R *dg = (const R *)d.dg;
  for (int k = 0; k < 12; k++) out[(size_t)k * d.nt + c] = (double)dg[k * d.cs + j];
}

// caller order (stride nt) <-> device order (stride cs)
__global__ void k_gather(int nt, int cs, int nvar, const int *perm, const double *src, double *dst) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nt) return;
  int c = perm[j];
  for (int v = 0; v < nvar; v++) dst[(size_t)v * cs + j] = src ? src[(size_t)v * nt + c] : 0.0;
}
__global__ void k_scatter(int nt, int cs, int nvar, const int *perm, const double *src, double *dst) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nt) return;
  int c = perm[j];
  for (int v = 0; v < nvar; v++) dst[(size_t)v * nt + c] = src[(size_t)v * cs + j];
}
// the status word of one pipelined item, kept before the next item resets it
__global__ void k_status_or(const int *st, int *acc) { *acc |= *st; }

// FMA-chain throughput probe for the roofline denominators (measurement only)
template <typename T>
__global__ void k_fma_probe(T *out, int iters, T a, T b) {
  T acc[8];
#pragma unroll
  for (int i = 0; i < 8; i++) acc[i] = (T)(threadIdx.x + i);
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int i = 0; i < 8; i++) acc[i] = acc[i] * a + b;
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < 8; i++) s += acc[i];
  if (s == (T)-1.2345) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// ------------------------------------------------------------- workspace
struct Carver {
  char *base;
  size_t off = 0;
  template <typename T> T *take(size_t n) {
    off = (off + 255) & ~size_t(255);
    T *p = base ? (T *)(base + off) : nullptr;
    off += n * sizeof(T);
    return p;
  }
};

}  // namespace

struct gks2l_ctx {
  Prep prep;
  gks2l_params par{};
  std::vector<double> bvert;
  bool has_b = false, bound = false, has_state = false;
  size_t rsize = 8;
  int cs = 0;                  // padded cell stride
  char *ws = nullptr;
  size_t ws_bytes = 0;
  cudaStream_t stream = nullptr;
  Dev d{};
  int *d_perm = nullptr;
  double *d_tend = nullptr;
  double *d_stage = nullptr;   // 18 * nt staging for permutations
  int nchunk = 0;              // reference-level reduction: chunks of one instance's cells
  int *d_chunk = nullptr;      // [nchunk][2] first and end cell of each chunk
  int *d_inst_chunk = nullptr; // [ninst + 1] first chunk of each instance
  double *d_refpart = nullptr; // [nchunk][3] the chunks' sums
  bool has_mlp = false;
  int n_sm = 1;                // SMs of the bound device
  cudaStream_t side = nullptr; // second stream for the gate (created with the network)
  int shape[4] = {1, 1, 1, 0}; // launch shapes of the interface, edge and update kernels; gate variant
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int phase = 0;
  int64_t stages = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  // pipelined host I/O (gks2l_run_items, allocated on first use): two input
  // and two output staging buffers of 18 * nt doubles, a copy stream for each
  // direction and the events that hand the buffers between the streams
  double *io_in[2] = {nullptr, nullptr}, *io_out[2] = {nullptr, nullptr};
  int *d_status_any = nullptr;
  cudaStream_t io_h2d = nullptr, io_d2h = nullptr;
  cudaEvent_t ev_in_ready[2] = {}, ev_in_free[2] = {}, ev_out_ready[2] = {}, ev_out_free[2] = {};
  std::string err;
};

namespace {

size_t layout(gks2l_ctx *c, char *base) {
  const Prep &P = c->prep;
  const size_t nt = P.nt, ne = P.ne, ni = P.ninst, rs = c->rsize;
  const size_t cs = (nt + TW - 1) / TW * TW + TW;   // one spare tile past the last one read
  c->cs = (int)cs;
  Carver k{base};
  Dev &d = c->d;
  d.nt = P.nt; d.ne = P.ne; d.ninst = P.ninst; d.cs = (int)cs;
  d.inst = k.take<int>(nt);
  d.area = k.take<double>(nt);
  d.hs = k.take<double>(nt);
  d.dX = k.take<double>(nt);
  d.hsR = k.take<char>(rs * nt);
  d.ihsR = k.take<char>(rs * nt);
  d.epsA = k.take<char>(rs * nt);
  d.bgR = k.take<char>(rs * 2 * cs);
  d.bmean = k.take<double>(nt);
  d.bgx = k.take<double>(nt);
  d.bgy = k.take<double>(nt);
  d.st_cell = k.take<int>(kSlots * cs);
  d.st_xf = k.take<int8_t>(kSlots * cs);
  d.ops = k.take<char>((cs / TW) * (rs == 4 ? TileLayout<float>::TILE : TileLayout<double>::TILE));
  d.plane = k.take<char>(rs * 6 * cs);
  d.cedge = k.take<int>(3 * cs);
  d.fsl = k.take<double>(3 * cs);
  d.fslR = k.take<char>(rs * 3 * cs);
  d.inst_first = k.take<int>(ni + 1);
  d.avg = k.take<double>(6 * cs);
  d.dq = k.take<char>(rs * 6 * cs);
  d.dg = k.take<char>(rs * 12 * cs);
  d.hrefc = k.take<char>(rs * nt);
  d.Wn = k.take<double>(6 * cs);
  d.Ln = k.take<double>(6 * cs);
  d.Ltn = k.take<double>(6 * cs);
  d.incR = k.take<char>(rs * 4 * cs);
  d.srec = k.take<char>(rs * 2 * NREC * cs);
  d.omg = k.take<char>(rs * 2 * cs);
  d.mlp = k.take<MlpDev>(1);
  d.gate_mask = k.take<unsigned>(cs / TW);
  d.gate_next = k.take<unsigned>(cs / TW);
  d.pos_flag = k.take<unsigned char>(2 * cs);
  d.pos_hbar = k.take<char>(rs * 2 * cs);
  d.wdev = k.take<float>(6 * cs);
  d.eL = k.take<int>(ne);
  d.eR = k.take<int>(ne);
  d.exf = k.take<int8_t>(ne);
  d.en = k.take<char>(rs * 2 * ne);
  d.eb0 = k.take<double>(ne);
  d.eb1 = k.take<double>(ne);
  d.exiL = k.take<char>(rs * 4 * ne);
  d.exiR = k.take<char>(rs * 4 * ne);
  d.hrefe = k.take<char>(rs * 2 * ne);
  d.hc = k.take<char>(rs * 2 * ne);
  d.wl = k.take<int>(2 * ne);
  d.wl_count = k.take<int>(1);
  d.eF = k.take<char>(rs * 6 * ne);
  d.eFt = k.take<char>(rs * 6 * ne);
  d.eFm = k.take<double>(2 * ne);
  d.eFtm = k.take<double>(2 * ne);
  d.eO = k.take<char>(rs * 4 * ne);
  d.eWt = k.take<char>(rs * 6 * ne);
  d.eWn = k.take<char>(rs * 6 * ne);
  d.ref = k.take<double>(2 * ni);
  d.refR = k.take<char>(rs * 2 * ni);
  d.dt = k.take<double>(ni);
  d.dtR = k.take<char>(rs * ni);
  d.t = k.take<double>(ni);
  d.dtbits = k.take<unsigned long long>(ni);
  d.mass = k.take<double>(2 * ni);
  d.status = k.take<int>(1);
  d.gate_count = k.take<unsigned long long>(2);
  d.xf = k.take<double>(4 * kMaxXf);
  c->d_perm = k.take<int>(nt);
  c->d_tend = k.take<double>(1);
  c->d_stage = k.take<double>(18 * nt);
  // at most one chunk per instance plus one per REF_CHUNK cells (the sizes
  // only: the workspace size is asked for before the instances are known)
  const size_t max_chunks = ni + nt / REF_CHUNK + 1;
  c->d_chunk = k.take<int>(2 * max_chunks);
  c->d_inst_chunk = k.take<int>(ni + 1);
  c->d_refpart = k.take<double>(3 * max_chunks);
  return k.off + 256;
}

#define CK(x)                                                                              \
  do {                                                                                     \
    cudaError_t e_ = (x);                                                                  \
    if (e_ != cudaSuccess) {                                                               \
      c->err = std::string(#x) + ": " + cudaGetErrorString(e_);                            \
      return GKS2L_ECUDA;                                                                  \
    }                                                                                      \
  } while (0)

template <typename T>
int upload(gks2l_ctx *c, const void *dst, const std::vector<T> &src) {
  if (src.empty()) return 0;
  CK(cudaMemcpyAsync((void *)dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));   // src may be a temporary
  return 0;
}
// [rows][nt] host array -> [rows][cs] device array of type T (padding zeroed)
template <typename T, typename S>
int upload_rows(gks2l_ctx *c, const void *dst, const std::vector<S> &src, int rows) {
  const size_t nt = c->prep.nt, cs = c->cs;
  std::vector<T> tmp(rows * cs, (T)0);
  for (int r = 0; r < rows; r++)
    for (size_t j = 0; j < nt; j++) tmp[r * cs + j] = (T)src[r * nt + j];
  return upload(c, dst, tmp);
}
// a double host array in the form's precision (single row or [rows][cs])
int upload_form(gks2l_ctx *c, const void *dst, const std::vector<double> &src, int rows, bool padded) {
  if (padded) return c->rsize == 4 ? upload_rows<float>(c, dst, src, rows) : upload_rows<double>(c, dst, src, rows);
  if (c->rsize == 4) return upload(c, dst, std::vector<float>(src.begin(), src.end()));
  return upload(c, dst, src);
}

// the reconstruction's operator rows, tile by tile in the layout k_recon
// copies (TileLayout), in the form's precision; packed on the host a batch of
// tiles at a time (cells past the end are zero)
template <typename R>
int upload_tiles(gks2l_ctx *c) {
  using T = TileLayout<R>;
  const Prep &P = c->prep;
  const size_t nt = P.nt, ntile = c->cs / TW, batch = 1024;
  std::vector<unsigned char> buf(batch * T::TILE);
  for (size_t t0 = 0; t0 < ntile; t0 += batch) {
    const size_t nb = std::min(batch, ntile - t0);
    std::fill(buf.begin(), buf.end(), (unsigned char)0);
    for (size_t t = 0; t < nb; t++) {
      unsigned char *b = buf.data() + t * T::TILE;
      R *lsq = (R *)(b + T::LSQ), *mm = (R *)(b + T::MM), *p1 = (R *)(b + T::P1), *bq = (R *)(b + T::BQ);
      int *st = (int *)(b + T::ST);
      int8_t *sx = (int8_t *)(b + T::SX);
      for (int i = 0; i < TW; i++) {
        const size_t j = (t0 + t) * TW + i;
        if (j >= nt) break;
        for (int r = 0; r < kCoef * kCols; r++) lsq[r * TW + i] = (R)P.lsq[r * nt + j];
        for (int r = 0; r < 7; r++) mm[r * TW + i] = (R)P.mmean[r * nt + j];
        for (int r = 0; r < kSlots; r++) {
          st[r * TW + i] = P.st_cell[r * nt + j];
          sx[r * TW + i] = P.st_xf[r * nt + j];
        }
        for (int r = 0; r < 30; r++) p1[r * TW + i] = (R)P.p1op[r * nt + j];
        for (int r = 0; r < kBeta; r++) bq[r * TW + i] = (R)P.bq[r * nt + j];
      }
    }
    CK(cudaMemcpyAsync((char *)c->d.ops + t0 * T::TILE, buf.data(), nb * T::TILE, cudaMemcpyHostToDevice,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  return 0;
}

inline unsigned blocks(size_t n, unsigned b) { return (unsigned)((n + b - 1) / b); }

int upload_bathymetry(gks2l_ctx *c) {
  std::vector<double> bm, bx, by, e0, e1;
  bathymetry(c->prep, c->has_b ? c->bvert.data() : nullptr, bm, bx, by, e0, e1);
  std::vector<double> bg(2 * (size_t)c->prep.nt);
  std::copy(bx.begin(), bx.end(), bg.begin());
  std::copy(by.begin(), by.end(), bg.begin() + c->prep.nt);
  int rc;
  if ((rc = upload(c, c->d.bmean, bm)) || (rc = upload(c, c->d.bgx, bx)) || (rc = upload(c, c->d.bgy, by)) ||
      (rc = upload(c, c->d.eb0, e0)) || (rc = upload(c, c->d.eb1, e1)) ||
      (rc = upload_form(c, c->d.bgR, bg, 2, true)))
    return rc;
  return 0;
}

Par make_par(const gks2l_ctx *c) {
  Par p;
  p.g = c->par.g; p.chi = c->par.chi; p.cfl = c->par.cfl;
  p.eps = c->par.eps; p.eps_num = c->par.eps_num;
  p.gam_hi = c->par.weno_gamma_hi; p.weno_eps = c->par.weno_eps;
  p.gf = (float)p.g; p.chif = (float)p.chi; p.epsf = (float)p.eps; p.eps_numf = (float)p.eps_num;
  p.gam_hif = (float)p.gam_hi;
  p.use_gate = (c->par.indicator == GKS2L_INDICATOR_MLP && c->has_mlp) ? 1 : 0;
  p.harvest = 0;
  p.logit_out = nullptr;
  p.all_active = 0;
  p.staging_polls = c->par.staging_poll_limit;
  p.pos_floor = c->par.positivity_floor;
  return p;
}


// gate variants: kernel (variant % 4): 0 mma.sync warp tiles, 1-3 tcgen05 CTA
// tiles at 1, 2 and 4 times the blocks per SM; placement (variant / 4 % 2):
// beside the edge kernels or the reconstruction; edge path (variant / 8):
// the fused pass or the plain kernels
constexpr int kGateKernels = 4, kGateVariants = 4 * kGateKernels;
inline int gate_kernel(int v) { return v % kGateKernels; }
inline bool gate_beside_recon(int v) { return (v / kGateKernels) % 2 == 1; }
inline bool gate_plain_edges(int v) { return v >= 2 * kGateKernels; }

// the gate in its chosen kernel: 0: warp tiles of 32 cells on mma.sync,
// 1: CTA tiles of 128 cells on tcgen05 with tensor-memory accumulators,
// 2 and 3: the same with two and four times the CTAs per SM (more gathers
// in flight; at four, eight CTAs fill an SM's registers and hold 256 of its
// 512 tensor-memory columns)
template <typename R>
void launch_gate(gks2l_ctx *c, const Par &p, cudaStream_t st) {
  const int kernel = gate_kernel(c->shape[3]);
  const unsigned per_sm = GATE_BLOCKS_PER_SM * (kernel == 3 ? 4 : kernel == 2 ? 2 : 1);
  const unsigned nb = std::min(blocks(c->d.nt, 4 * TW), (unsigned)(c->n_sm * per_sm));
  if (kernel >= 1) k_gate_tc<R><<<nb, GATE_TC_M, 0, st>>>(c->d, p);
  else k_gate<R><<<nb, 128, 0, st>>>(c->d, p);
}

template <typename R>
void launch_recon(gks2l_ctx *c, const Par &p) {
  const Dev &d = c->d;
  if (p.pos_floor > 0) k_recon<R, true><<<blocks(d.nt, TW), dim3(TW, 6), recon_smem<R>(), c->stream>>>(d, p);
  else k_recon<R><<<blocks(d.nt, TW), dim3(TW, 6), recon_smem<R>(), c->stream>>>(d, p);
}

// launch shapes the autotuner chooses from: 0: 64 threads, 1: 128 threads,
// 2: 256 threads (registers as the compiler likes), 3: 128 threads held to
// 64 registers (eight blocks per SM), 4: 128 threads held to 128 registers
constexpr int kShapes = 5;

#define GKS2L_SHAPE_SWITCH(cfg, KERNEL, n, st, ...)                                          \
  switch (cfg) {                                                                           \
    case 0: KERNEL<R, 64><<<blocks(n, 64), 64, 0, st>>>(__VA_ARGS__); break;                \
    case 2: KERNEL<R, 256><<<blocks(n, 256), 256, 0, st>>>(__VA_ARGS__); break;             \
    case 3: KERNEL##_r64<R><<<blocks(n, 128), 128, 0, st>>>(__VA_ARGS__); break;            \
    case 4: KERNEL##_r128<R><<<blocks(n, 128), 128, 0, st>>>(__VA_ARGS__); break;           \
    default: KERNEL<R, 128><<<blocks(n, 128), 128, 0, st>>>(__VA_ARGS__); break;            \
  }

template <typename R>
void launch_iface(gks2l_ctx *c, cudaStream_t st) {
  const size_t n = 2 * (size_t)c->d.ne;
  GKS2L_SHAPE_SWITCH(c->shape[0], k_iface, n, st, c->d)
}

template <typename R>
void launch_edge(gks2l_ctx *c, const Par &p, int stage, cudaStream_t st) {
  const size_t n = 4 * (size_t)c->d.ne;
  if (p.pos_floor > 0) {
    k_edge_pos<R><<<blocks(n, 128), 128, 0, st>>>(c->d, p, stage);
    return;
  }
  GKS2L_SHAPE_SWITCH(c->shape[1], k_edge, n, st, c->d, p, stage)
}

// gated runs: interface levels and edge solution fused, then the deferred units
template <typename R>
void launch_edge_fused(gks2l_ctx *c, const Par &p, int stage, cudaStream_t st) {
  const size_t n = 4 * (size_t)c->d.ne;
  cudaMemsetAsync(c->d.wl_count, 0, sizeof(int), st);
  GKS2L_SHAPE_SWITCH(c->shape[1], k_edgef, n, st, c->d, p, stage)
}
template <typename R>
void launch_edge_deferred(gks2l_ctx *c, const Par &p, int stage, cudaStream_t st) {
  k_edge_deferred<R><<<c->n_sm * DEFER_BLOCKS_PER_SM, 128, 0, st>>>(c->d, p, stage);
}

template <typename R>
void launch_update(gks2l_ctx *c, const Par &p, int stage, cudaStream_t st) {
  const size_t n = (size_t)c->d.nt;
  GKS2L_SHAPE_SWITCH(c->shape[2], k_update, n, st, c->d, p, stage)
}

// With the gate on, the interface levels and the edge solution run as one
// fused pass plus the deferred edges (gate variants 0-7), or as the plain
// interface and edge kernels (8-15), which a gate that calls few cells
// smooth leaves faster.
inline bool fused_edges(const gks2l_ctx *c, const Par &p) {
  return p.use_gate && !gate_plain_edges(c->shape[3]) && !(p.pos_floor > 0);
}

// the gate on the second stream, from this point of the main stream on
template <typename R>
void fork_gate(gks2l_ctx *c, const Par &p) {
  cudaEventRecord(c->ev_fork, c->stream);
  cudaStreamWaitEvent(c->side, c->ev_fork, 0);
  launch_gate<R>(c, p, c->side);
  cudaEventRecord(c->ev_join, c->side);
}

template <typename R>
void launch_stage(gks2l_ctx *c, int stage) {
  Par p = make_par(c);
  // The gate for the next stage reads this stage's state, which only
  // k_update replaces, and writes its mask to a second buffer: it runs beside
  // the reconstruction or beside the edge kernels (the variant's placement)
  // and joins before k_update, which copies the mask over.
  const bool gate_early = p.use_gate && gate_beside_recon(c->shape[3]);
  if (gate_early) fork_gate<R>(c, p);
  launch_recon<R>(c, p);
  if (p.use_gate && !gate_early) fork_gate<R>(c, p);
  if (fused_edges(c, p)) {
    launch_edge_fused<R>(c, p, stage, c->stream);
    launch_edge_deferred<R>(c, p, stage, c->stream);
  } else {
    launch_iface<R>(c, c->stream);
    launch_edge<R>(c, p, stage, c->stream);
  }
  if (p.use_gate) cudaStreamWaitEvent(c->stream, c->ev_join, 0);
  launch_update<R>(c, p, stage, c->stream);
}

void launch_stage_any(gks2l_ctx *c, int stage) {
  if (c->par.precision == GKS2L_FP32) launch_stage<float>(c, stage);
  else launch_stage<double>(c, stage);
}

void launch_step_begin(gks2l_ctx *c) {
  Par p = make_par(c);
  if (c->par.precision == GKS2L_FP32)
    k_step_begin<float><<<blocks(c->d.ninst, 128), 128, 0, c->stream>>>(c->d, p, c->d_tend);
  else
    k_step_begin<double><<<blocks(c->d.ninst, 128), 128, 0, c->stream>>>(c->d, p, c->d_tend);
}

void drop_graph(gks2l_ctx *c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->graph) cudaGraphDestroy(c->graph);
  c->gexec = nullptr;
  c->graph = nullptr;
}

int ensure_graph(gks2l_ctx *c) {
  if (c->gexec || !c->stream) return 0;
  CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  launch_step_begin(c);
  launch_stage_any(c, 1);
  launch_stage_any(c, 2);
  cudaError_t e = cudaStreamEndCapture(c->stream, &c->graph);
  if (e != cudaSuccess) {
    c->err = std::string("graph capture: ") + cudaGetErrorString(e);
    c->graph = nullptr;
    return GKS2L_ECUDA;
  }
  CK(cudaGraphInstantiate(&c->gexec, c->graph, 0));
  return 0;
}

// a staging timeout first: the stages after it computed from stale records,
// so the non-finite values or depths they may show are its consequence
int status_code(int st) {
  if (st & (ST_TIMEOUT | ST_COPY_LOST)) return GKS2L_ETIMEOUT;
  if (st & 2) return GKS2L_ENONFINITE;
  if (st & 1) return GKS2L_ENEGDEPTH;
  return 0;
}

int check_status(gks2l_ctx *c) {
  int st = 0;
  CK(cudaMemcpyAsync(&st, c->d.status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return status_code(st);
}

// Reference levels per instance: area-weighted means of h2 and eta1 = h1 + B
// of the state in device order (host, deterministic), rounded to 2^-32.
// after d.avg (device order) is set and the caller's gradients sit at
// grad_caller (device memory, caller order, or NULL): references, mirrors,
// reference depths on the edges, counters, CFL ratio and masses
int after_state(gks2l_ctx *c, const double *grad_caller) {
  // the reference levels on the device (no copy of the state to the host)
  k_ref_partial<<<c->nchunk, REF_THREADS, 0, c->stream>>>(c->d, c->d_chunk, c->d_refpart);
  Par p = make_par(c);
  if (c->par.precision == GKS2L_FP32) {
    k_ref_final<float><<<blocks(c->d.ninst, 128), 128, 0, c->stream>>>(c->d, c->d_inst_chunk, c->d_refpart);
    k_mirrors<float><<<blocks(c->d.nt, 128), 128, 0, c->stream>>>(c->d, c->d_perm, grad_caller);
    k_edge_ref<float><<<blocks(c->d.ne, 128), 128, 0, c->stream>>>(c->d);
  } else {
    k_ref_final<double><<<blocks(c->d.ninst, 128), 128, 0, c->stream>>>(c->d, c->d_inst_chunk, c->d_refpart);
    k_mirrors<double><<<blocks(c->d.nt, 128), 128, 0, c->stream>>>(c->d, c->d_perm, grad_caller);
    k_edge_ref<double><<<blocks(c->d.ne, 128), 128, 0, c->stream>>>(c->d);
  }
  k_reset_stats<<<blocks(c->d.ninst, 128), 128, 0, c->stream>>>(c->d);
  CK(cudaMemsetAsync(c->d.t, 0, sizeof(double) * c->d.ninst, c->stream));
  CK(cudaMemsetAsync(c->d.dt, 0, sizeof(double) * c->d.ninst, c->stream));
  CK(cudaMemsetAsync(c->d.status, 0, sizeof(int), c->stream));
  CK(cudaMemsetAsync(c->d.gate_count, 0, 2 * sizeof(unsigned long long), c->stream));
  if (c->par.precision == GKS2L_FP32) k_cfl<float><<<blocks(c->d.nt, 128), 128, 0, c->stream>>>(c->d, p);
  else k_cfl<double><<<blocks(c->d.nt, 128), 128, 0, c->stream>>>(c->d, p);
  if (p.use_gate) {
    // the gate's decisions on the state just set serve the first
    // reconstruction (every cell counts as active: no dt is known yet)
    Par pg = p;
    pg.all_active = 1;
    if (c->par.precision == GKS2L_FP32) launch_gate<float>(c, pg, c->stream);
    else launch_gate<double>(c, pg, c->stream);
    CK(cudaMemcpyAsync(c->d.gate_mask, c->d.gate_next, (c->cs / TW) * sizeof(unsigned), cudaMemcpyDeviceToDevice,
                       c->stream));
  } else {
    // no gate decisions: the first reconstruction is the plain one
    CK(cudaMemsetAsync(c->d.gate_mask, 0, (c->cs / TW) * sizeof(unsigned), c->stream));
  }
  CK(cudaGetLastError());
  c->phase = 0;
  c->stages = 0;
  c->has_state = true;
  return 0;
}

int create_impl(int n, const gks2l_mesh *meshes, const gks2l_params *params, gks2l_ctx **out) {
  if (!meshes || !out || n <= 0) return GKS2L_EINVAL;
  gks2l_ctx *c = new gks2l_ctx();
  if (params) c->par = *params;
  else gks2l_default_params(&c->par);
  if (!(c->par.g > 0) || !(c->par.cfl > 0) || !(c->par.eps > 0) || c->par.eps_num < 0 || !(c->par.chi > 0) ||
      !(c->par.weno_gamma_hi > 0 && c->par.weno_gamma_hi <= 1) || c->par.weno_eps < 0 ||
      (c->par.precision != GKS2L_FP64 && c->par.precision != GKS2L_FP32) || c->par.staging_poll_limit < 0 ||
      !(c->par.positivity_floor >= 0 && c->par.positivity_floor < 1)) {
    delete c;
    return GKS2L_EINVAL;
  }
  c->rsize = c->par.precision == GKS2L_FP32 ? 4 : 8;
  int rc = prepare(n, meshes, c->prep, c->err);
  if (rc) {
    fprintf(stderr, "gks2l: %s\n", c->err.c_str());
    delete c;
    return rc;
  }
  *out = c;
  return GKS2L_OK;
}

}  // namespace

extern "C" {

int gks2l_default_params(gks2l_params *p) {
  if (!p) return GKS2L_EINVAL;
  p->g = 9.81;
  p->chi = 1.0;
  p->cfl = 0.5;
  p->eps = 0.05;
  p->eps_num = 5.0;
  p->weno_gamma_hi = 0.85;
  p->weno_eps = 1.0;
  p->precision = GKS2L_FP64;
  p->indicator = GKS2L_INDICATOR_OFF;
  p->indicator_threshold = 0.5f;
  p->staging_poll_limit = 0;
  p->positivity_floor = 0;
  return GKS2L_OK;
}

int gks2l_create(const gks2l_mesh *mesh, const gks2l_params *params, gks2l_ctx **out) {
  return create_impl(1, mesh, params, out);
}

int gks2l_create_ensemble(int32_t n, const gks2l_mesh *meshes, const gks2l_params *params, gks2l_ctx **out) {
  return create_impl(n, meshes, params, out);
}

int gks2l_workspace_bytes(const gks2l_ctx *ctx, size_t *bytes) {
  if (!ctx || !bytes) return GKS2L_EINVAL;
  gks2l_ctx tmp;
  tmp.prep.nt = ctx->prep.nt;
  tmp.prep.ne = ctx->prep.ne;
  tmp.prep.ninst = ctx->prep.ninst;
  tmp.rsize = ctx->rsize;
  *bytes = layout(&tmp, nullptr);
  return GKS2L_OK;
}

int gks2l_bind(gks2l_ctx *c, void *d_workspace, size_t bytes, void *stream) {
  if (!c || !d_workspace) return GKS2L_EINVAL;
  if (((uintptr_t)d_workspace & 255) != 0) return GKS2L_EINVAL;
  size_t need = layout(c, nullptr);
  if (bytes < need) return GKS2L_ESPACE;
  drop_graph(c);
  c->ws = (char *)d_workspace;
  c->ws_bytes = bytes;
  c->stream = (cudaStream_t)stream;
  layout(c, c->ws);
  CK(cudaMemsetAsync(c->ws, 0, need, c->stream));   // padding rows and tiles start at zero
  const Prep &P = c->prep;
  const int nt = P.nt;
  std::vector<double> fsl(3 * (size_t)nt), en(2 * (size_t)P.ne), ihs(nt), epsA(nt);
  for (int j = 0; j < nt; j++) {
    for (int f = 0; f < 3; f++) {
      int ce = P.cedge[f * nt + j];
      int e = ce >= 0 ? ce : ~ce;
      fsl[f * nt + j] = (ce >= 0 ? 1.0 : -1.0) * P.elen[e] / P.area[j];
    }
    ihs[j] = 1.0 / P.hs[j];
    epsA[j] = c->par.weno_eps * P.area[j];
  }
  for (int e = 0; e < P.ne; e++) { en[e] = P.en0[e]; en[P.ne + e] = P.en1[e]; }
  std::vector<double> xf(4 * kMaxXf, 0.0);
  std::copy(P.xf.begin(), P.xf.end(), xf.begin());
  int rc;
  if ((rc = upload(c, c->d.inst, P.inst)) || (rc = upload(c, c->d.area, P.area)) ||
      (rc = upload(c, c->d.hs, P.hs)) || (rc = upload(c, c->d.dX, P.dX)) ||
      (rc = upload_rows<int>(c, c->d.st_cell, P.st_cell, kSlots)) ||
      (rc = upload_rows<int8_t>(c, c->d.st_xf, P.st_xf, kSlots)) ||
      (rc = upload_rows<int>(c, c->d.cedge, P.cedge, 3)) || (rc = upload_rows<double>(c, c->d.fsl, fsl, 3)) ||
      (rc = upload_form(c, c->d.fslR, fsl, 3, true)) ||
      (rc = upload(c, c->d.inst_first, P.inst_first)) || (rc = upload(c, c->d.eL, P.eL)) ||
      (rc = upload(c, c->d.eR, P.eR)) || (rc = upload(c, c->d.exf, P.exf)) || (rc = upload(c, c->d.xf, xf)) ||
      (rc = upload(c, c->d_perm, P.perm)) ||
      (rc = c->rsize == 4 ? upload_tiles<float>(c) : upload_tiles<double>(c)) ||
      (rc = upload_form(c, c->d.plane, P.plane, 6, true)) ||
      (rc = upload_form(c, c->d.hsR, P.hs, 1, false)) || (rc = upload_form(c, c->d.ihsR, ihs, 1, false)) ||
      (rc = upload_form(c, c->d.epsA, epsA, 1, false)) || (rc = upload_form(c, c->d.exiL, P.exiL, 1, false)) ||
      (rc = upload_form(c, c->d.exiR, P.exiR, 1, false)) || (rc = upload_form(c, c->d.en, en, 1, false)))
    return rc;
  {
    std::vector<int> ch, ich(P.ninst + 1);
    for (int i = 0; i < P.ninst; i++) {
      ich[i] = (int)(ch.size() / 2);
      const int j0 = P.inst_first[i], j1 = P.inst_first[i + 1];
      int j = j0;
      do {
        const int e = std::min(j1, j + REF_CHUNK);
        ch.push_back(j);
        ch.push_back(e);
        j = e;
      } while (j < j1);
    }
    ich[P.ninst] = (int)(ch.size() / 2);
    c->nchunk = (int)(ch.size() / 2);
    if ((size_t)c->nchunk > (size_t)P.ninst + (size_t)P.nt / REF_CHUNK + 1) {
      c->err = "reference chunk table larger than its slice";
      return GKS2L_EINVAL;
    }
    if ((rc = upload(c, c->d_chunk, ch)) || (rc = upload(c, c->d_inst_chunk, ich))) return rc;
  }
  {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, dev));
  }
  CK(cudaFuncSetAttribute(k_recon<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, recon_smem<float>()));
  CK(cudaFuncSetAttribute(k_recon<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, recon_smem<double>()));
  CK(cudaFuncSetAttribute(k_recon<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, recon_smem<float>()));
  CK(cudaFuncSetAttribute(k_recon<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          recon_smem<double>()));
  c->bound = true;
  c->has_state = false;
  return upload_bathymetry(c);
}

int gks2l_set_bathymetry(gks2l_ctx *c, const double *b_vert) {
  if (!c || !b_vert) return GKS2L_EINVAL;
  c->bvert.assign(b_vert, b_vert + c->prep.nv);
  c->has_b = true;
  c->has_state = false;   // the level mirrors depend on B: set the state again
  if (c->bound) return upload_bathymetry(c);
  return GKS2L_OK;
}

int gks2l_set_state(gks2l_ctx *c, const double *avg, const double *grad) {
  if (!c || !avg) return GKS2L_EINVAL;
  if (!c->bound) return GKS2L_ESTATE;
  const size_t nt = c->prep.nt;
  CK(cudaMemcpyAsync(c->d_stage, avg, 6 * nt * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  if (grad) CK(cudaMemcpyAsync(c->d_stage + 6 * nt, grad, 12 * nt * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  k_gather<<<blocks(nt, 128), 128, 0, c->stream>>>((int)nt, c->cs, 6, c->d_perm, c->d_stage, c->d.avg);
  CK(cudaGetLastError());
  int rc = after_state(c, grad ? c->d_stage + 6 * nt : nullptr);
  if (rc) return rc;
  CK(cudaStreamSynchronize(c->stream));   // the host arrays may be released after return
  return GKS2L_OK;
}

int gks2l_set_state_device(gks2l_ctx *c, const double *d_avg, const double *d_grad) {
  if (!c || !d_avg) return GKS2L_EINVAL;
  if (!c->bound) return GKS2L_ESTATE;
  const size_t nt = c->prep.nt;
  k_gather<<<blocks(nt, 128), 128, 0, c->stream>>>((int)nt, c->cs, 6, c->d_perm, d_avg, c->d.avg);
  CK(cudaGetLastError());
  return after_state(c, d_grad);
}

constexpr int kAdvanceCheck = 32;   // steps between end-time checks in gks2l_advance

int gks2l_advance(gks2l_ctx *c, int32_t n_stages, double t_end, double *t_out) {
  if (!c || n_stages < 0) return GKS2L_EINVAL;
  if (!c->bound || !c->has_state) return GKS2L_ESTATE;
  CK(cudaMemcpyAsync(c->d_tend, &t_end, sizeof(double), cudaMemcpyHostToDevice, c->stream));
  int left = n_stages;
  if (left > 0 && c->phase == 1) {
    launch_stage_any(c, 2);
    c->phase = 0;
    left--;
    c->stages++;
  }
  int steps = left / 2;
  bool arrived = false;
  if (steps > 0) {
    int rc = ensure_graph(c);
    if (rc) return rc;
    // with an end time, every kAdvanceCheck steps the instances' times are
    // read back and the call stops once all have reached it (later steps
    // would change nothing)
    std::vector<double> tv(t_end > 0 ? c->prep.ninst : 0);
    const double tol = 1e-12 * std::max(1.0, std::fabs(t_end));
    for (int s = 0; s < steps; s++) {
      if (c->gexec) {
        CK(cudaGraphLaunch(c->gexec, c->stream));
      } else {
        launch_step_begin(c);
        launch_stage_any(c, 1);
        launch_stage_any(c, 2);
      }
      c->stages += 2;
      if (t_end > 0 && (s + 1) % kAdvanceCheck == 0 && s + 1 < steps) {
        CK(cudaMemcpyAsync(tv.data(), c->d.t, tv.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        arrived = true;
        for (double t : tv)
          if (t_end - t > tol) arrived = false;
        if (arrived) break;
      }
    }
  }
  if (left % 2 && !arrived) {
    launch_step_begin(c);
    launch_stage_any(c, 1);
    c->phase = 1;
    c->stages++;
  }
  CK(cudaGetLastError());
  if (t_out) {
    CK(cudaMemcpyAsync(t_out, c->d.t, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    return check_status(c);
  }
  return GKS2L_OK;
}

int gks2l_get_state(gks2l_ctx *c, double *avg, double *grad) {
  if (!c || !avg) return GKS2L_EINVAL;
  if (!c->bound || !c->has_state) return GKS2L_ESTATE;
  const size_t nt = c->prep.nt;
  k_scatter<<<blocks(nt, 128), 128, 0, c->stream>>>((int)nt, c->cs, 6, c->d_perm, c->d.avg, c->d_stage);
  if (c->par.precision == GKS2L_FP32)
    k_grad_out<float><<<blocks(nt, 128), 128, 0, c->stream>>>(c->d, c->d_perm, c->d_stage + 6 * nt);
  else
    k_grad_out<double><<<blocks(nt, 128), 128, 0, c->stream>>>(c->d, c->d_perm, c->d_stage + 6 * nt);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(avg, c->d_stage, 6 * nt * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  if (grad) CK(cudaMemcpyAsync(grad, c->d_stage + 6 * nt, 12 * nt * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return GKS2L_OK;
}

int gks2l_get_state_device(gks2l_ctx *c, double *d_avg, double *d_grad) {
  if (!c || !d_avg) return GKS2L_EINVAL;
  if (!c->bound || !c->has_state) return GKS2L_ESTATE;
  const size_t nt = c->prep.nt;
  k_scatter<<<blocks(nt, 128), 128, 0, c->stream>>>((int)nt, c->cs, 6, c->d_perm, c->d.avg, d_avg);
  if (d_grad) {
    if (c->par.precision == GKS2L_FP32)
      k_grad_out<float><<<blocks(nt, 128), 128, 0, c->stream>>>(c->d, c->d_perm, d_grad);
    else
      k_grad_out<double><<<blocks(nt, 128), 128, 0, c->stream>>>(c->d, c->d_perm, d_grad);
  }
  CK(cudaGetLastError());
  return GKS2L_OK;
}

// buffers, streams and events of gks2l_run_items, made on first use (each
// piece once, so a call that failed part way completes them on the next)
static int ensure_io(gks2l_ctx *c) {
  if (c->io_h2d) return 0;
  const size_t bytes = 18 * (size_t)c->prep.nt * sizeof(double);
  for (int b = 0; b < 2; b++) {
    if (!c->io_in[b]) CK(cudaMalloc((void **)&c->io_in[b], bytes));
    if (!c->io_out[b]) CK(cudaMalloc((void **)&c->io_out[b], bytes));
    for (cudaEvent_t *e : {&c->ev_in_ready[b], &c->ev_in_free[b], &c->ev_out_ready[b], &c->ev_out_free[b]})
      if (!*e) CK(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  }
  if (!c->d_status_any) CK(cudaMalloc((void **)&c->d_status_any, sizeof(int)));
  if (!c->io_d2h) CK(cudaStreamCreateWithFlags(&c->io_d2h, cudaStreamNonBlocking));
  CK(cudaStreamCreateWithFlags(&c->io_h2d, cudaStreamNonBlocking));
  return 0;
}

// n stages from a state just set (phase 0), enqueued without any host wait
static int enqueue_stages(gks2l_ctx *c, int n) {
  if (n / 2 > 0) {
    int rc = ensure_graph(c);
    if (rc) return rc;
  }
  for (int s = 0; s < n / 2; s++) {
    if (c->gexec) {
      CK(cudaGraphLaunch(c->gexec, c->stream));
    } else {
      launch_step_begin(c);
      launch_stage_any(c, 1);
      launch_stage_any(c, 2);
    }
    c->stages += 2;
  }
  if (n % 2) {
    launch_step_begin(c);
    launch_stage_any(c, 1);
    c->phase = 1;
    c->stages++;
  }
  CK(cudaGetLastError());
  return 0;
}

// the items' copies and stages, enqueued on the three streams
static int enqueue_items(gks2l_ctx *c, int32_t n_items, int32_t n_stages, const double *const *in_avg,
                         const double *const *in_grad, double *const *out_avg, double *const *out_grad) {
  int rc;
  const size_t nt = c->prep.nt, na = 6 * nt * sizeof(double), ng = 12 * nt * sizeof(double);
  // no end time: the steps' dt follow the CFL condition only
  CK(cudaMemsetAsync(c->d_tend, 0, sizeof(double), c->stream));
  CK(cudaMemsetAsync(c->d_status_any, 0, sizeof(int), c->stream));
  if (n_stages / 2 > 0 && (rc = ensure_graph(c))) return rc;
  for (int i = 0; i < n_items; i++) {
    const int b = i & 1;
    double *in = c->io_in[b], *out = c->io_out[b];
    const bool gi = in_grad && in_grad[i], go = out_grad && out_grad[i];
    // host -> device on the input stream, once item i - 2 has left the buffer
    if (i >= 2) CK(cudaStreamWaitEvent(c->io_h2d, c->ev_in_free[b], 0));
    CK(cudaMemcpyAsync(in, in_avg[i], na, cudaMemcpyHostToDevice, c->io_h2d));
    if (gi) CK(cudaMemcpyAsync(in + 6 * nt, in_grad[i], ng, cudaMemcpyHostToDevice, c->io_h2d));
    CK(cudaEventRecord(c->ev_in_ready[b], c->io_h2d));
    // the item on the compute stream: set, advance, keep its status
    CK(cudaStreamWaitEvent(c->stream, c->ev_in_ready[b], 0));
    if ((rc = gks2l_set_state_device(c, in, gi ? in + 6 * nt : nullptr))) return rc;
    CK(cudaEventRecord(c->ev_in_free[b], c->stream));
    if ((rc = enqueue_stages(c, n_stages))) return rc;
    k_status_or<<<1, 1, 0, c->stream>>>(c->d.status, c->d_status_any);
    // into the output buffer once item i - 2's result has left it, then
    // device -> host on the output stream
    if (i >= 2) CK(cudaStreamWaitEvent(c->stream, c->ev_out_free[b], 0));
    if ((rc = gks2l_get_state_device(c, out, go ? out + 6 * nt : nullptr))) return rc;
    CK(cudaEventRecord(c->ev_out_ready[b], c->stream));
    CK(cudaStreamWaitEvent(c->io_d2h, c->ev_out_ready[b], 0));
    CK(cudaMemcpyAsync(out_avg[i], out, na, cudaMemcpyDeviceToHost, c->io_d2h));
    if (go) CK(cudaMemcpyAsync(out_grad[i], out + 6 * nt, ng, cudaMemcpyDeviceToHost, c->io_d2h));
    CK(cudaEventRecord(c->ev_out_free[b], c->io_d2h));
  }
  return 0;
}

int gks2l_run_items(gks2l_ctx *c, int32_t n_items, int32_t n_stages, const double *const *in_avg,
                    const double *const *in_grad, double *const *out_avg, double *const *out_grad) {
  if (!c || n_items < 0 || n_stages < 0) return GKS2L_EINVAL;
  if (n_items > 0 && (!in_avg || !out_avg)) return GKS2L_EINVAL;
  for (int i = 0; i < n_items; i++)
    if (!in_avg[i] || !out_avg[i]) return GKS2L_EINVAL;
  if (!c->bound) return GKS2L_ESTATE;
  if (n_items == 0) return GKS2L_OK;
  int rc = ensure_io(c);
  if (rc) return rc;
  rc = enqueue_items(c, n_items, n_stages, in_avg, in_grad, out_avg, out_grad);
  // whatever was enqueued finishes before the caller's host arrays are
  // handed back, on the error path too
  const cudaError_t e[3] = {cudaStreamSynchronize(c->io_h2d), cudaStreamSynchronize(c->io_d2h),
                            cudaStreamSynchronize(c->stream)};
  if (rc) return rc;
  for (cudaError_t x : e) CK(x);
  int st = 0;
  CK(cudaMemcpyAsync(&st, c->d_status_any, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return status_code(st);
}

int gks2l_stats(gks2l_ctx *c, gks2l_stats_t *out) {
  if (!c || !out) return GKS2L_EINVAL;
  if (!c->bound || !c->has_state) return GKS2L_ESTATE;
  std::vector<double> mass(2 * c->prep.ninst);
  double t = 0, dt = 0;
  int st = 0;
  unsigned long long cnt[2] = {0, 0};
  CK(cudaMemsetAsync(c->d.mass, 0, mass.size() * sizeof(double), c->stream));
  k_mass<<<blocks(c->prep.nt, 128), 128, 0, c->stream>>>(c->d);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(mass.data(), c->d.mass, mass.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(&t, c->d.t, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(&dt, c->d.dt, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(&st, c->d.status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(cnt, c->d.gate_count, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  out->mass[0] = out->mass[1] = 0;
  for (int i = 0; i < c->prep.ninst; i++) {
    out->mass[0] += mass[2 * i];
    out->mass[1] += mass[2 * i + 1];
  }
  out->t = t;
  out->dt_last = dt;
  out->stages_done = c->stages;
  out->status = status_code(st);
  out->n_instances = c->prep.ninst;
  out->smooth_fraction = cnt[1] ? (double)cnt[0] / (double)cnt[1] : 0.0;
  return GKS2L_OK;
}

int gks2l_profile_kernels(gks2l_ctx *c, int32_t n_steps, double ms[6]) {
  if (!c || !ms || n_steps <= 0) return GKS2L_EINVAL;
  if (!c->bound || !c->has_state || c->phase != 0) return GKS2L_ESTATE;
  double zero = 0.0;
  CK(cudaMemcpyAsync(c->d_tend, &zero, sizeof(double), cudaMemcpyHostToDevice, c->stream));
  cudaEvent_t ev[8];
  for (int i = 0; i < 8; i++) CK(cudaEventCreate(&ev[i]));
  double acc[6] = {0, 0, 0, 0, 0, 0};
  Par p = make_par(c);
  const bool f32 = c->par.precision == GKS2L_FP32, fused = fused_edges(c, p);
  for (int s = 0; s < n_steps; s++) {
    CK(cudaEventRecord(ev[0], c->stream));
    launch_step_begin(c);
    CK(cudaEventRecord(ev[1], c->stream));
    for (int stage = 1; stage <= 2; stage++) {
      CK(cudaEventRecord(ev[2], c->stream));
      if (f32) launch_recon<float>(c, p);
      else launch_recon<double>(c, p);
      CK(cudaEventRecord(ev[3], c->stream));
      if (p.use_gate) {
        if (f32) launch_gate<float>(c, p, c->stream);
        else launch_gate<double>(c, p, c->stream);
      }
      // plain edge path: interface kernel between ev[7] and ev[4], edge
      // kernel up to ev[5]; fused path: fused kernel between ev[7] and ev[4] (reported as the
      // edge time), deferred pass up to ev[5] (reported in the interface slot)
      CK(cudaEventRecord(ev[7], c->stream));
      if (fused) {
        if (f32) launch_edge_fused<float>(c, p, stage, c->stream);
        else launch_edge_fused<double>(c, p, stage, c->stream);
      } else {
        if (f32) launch_iface<float>(c, c->stream);
        else launch_iface<double>(c, c->stream);
      }
      CK(cudaEventRecord(ev[4], c->stream));
      if (fused) {
        if (f32) launch_edge_deferred<float>(c, p, stage, c->stream);
        else launch_edge_deferred<double>(c, p, stage, c->stream);
      } else {
        if (f32) launch_edge<float>(c, p, stage, c->stream);
        else launch_edge<double>(c, p, stage, c->stream);
      }
      CK(cudaEventRecord(ev[5], c->stream));
      if (f32) launch_update<float>(c, p, stage, c->stream);
      else launch_update<double>(c, p, stage, c->stream);
      CK(cudaEventRecord(ev[6], c->stream));
      CK(cudaEventSynchronize(ev[6]));
      float t;
      CK(cudaEventElapsedTime(&t, ev[2], ev[3]));
      acc[0] += t;
      CK(cudaEventElapsedTime(&t, ev[3], ev[7]));
      acc[5] += t;
      CK(cudaEventElapsedTime(&t, ev[7], ev[4]));
      acc[fused ? 2 : 1] += t;
      CK(cudaEventElapsedTime(&t, ev[4], ev[5]));
      acc[fused ? 1 : 2] += t;
      CK(cudaEventElapsedTime(&t, ev[5], ev[6]));
      acc[3] += t;
    }
    float t0;
    CK(cudaEventElapsedTime(&t0, ev[0], ev[1]));
    acc[4] += t0;
  }
  CK(cudaGetLastError());
  for (int i = 0; i < 8; i++) cudaEventDestroy(ev[i]);
  for (int k = 0; k < 4; k++) ms[k] = acc[k] / (2.0 * n_steps);
  ms[4] = acc[4] / n_steps;
  ms[5] = acc[5] / (2.0 * n_steps);
  c->stages += 2 * n_steps;
  return GKS2L_OK;
}

int gks2l_set_launch_shapes(gks2l_ctx *c, const int32_t shapes[4]) {
  if (!c || !shapes) return GKS2L_EINVAL;
  for (int k = 0; k < 3; k++)
    if (shapes[k] < 0 || shapes[k] >= kShapes) return GKS2L_EINVAL;
  if (shapes[3] < 0 || shapes[3] >= kGateVariants) return GKS2L_EINVAL;
  for (int k = 0; k < 4; k++) c->shape[k] = shapes[k];
  drop_graph(c);
  return GKS2L_OK;
}

int gks2l_autotune(gks2l_ctx *c, int32_t n_steps, int32_t shapes[4]) {
  if (!c || !shapes || n_steps <= 0) return GKS2L_EINVAL;
  if (!c->bound || !c->has_state || c->phase != 0) return GKS2L_ESTATE;
  double best[3] = {INFINITY, INFINITY, INFINITY};
  int pick[3] = {c->shape[0], c->shape[1], c->shape[2]};
  for (int b = 0; b < kShapes; b++) {
    for (int k = 0; k < 3; k++) c->shape[k] = b;
    double ms[6];
    int rc = gks2l_profile_kernels(c, n_steps, ms);
    if (rc) return rc;
    // ms: reconstruction, interface, edge, update, ...
    for (int k = 0; k < 3; k++)
      if (ms[1 + k] < best[k]) {
        best[k] = ms[1 + k];
        pick[k] = b;
      }
  }
  for (int k = 0; k < 3; k++) c->shape[k] = shapes[k] = pick[k];
  drop_graph(c);
  // the gate runs beside other kernels on a second stream, so its variant is
  // chosen by whole steps (captured graphs, CUDA events), not by its own time
  shapes[3] = c->shape[3];
  if (c->par.indicator == GKS2L_INDICATOR_MLP && c->has_mlp) {
    double best_g = INFINITY;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    double zero = 0.0;
    CK(cudaMemcpyAsync(c->d_tend, &zero, sizeof(double), cudaMemcpyHostToDevice, c->stream));
    for (int v = 0; v < kGateVariants; v++) {
      c->shape[3] = v;
      drop_graph(c);
      int rc = ensure_graph(c);
      if (rc) return rc;
      CK(cudaGraphLaunch(c->gexec, c->stream));   // the first step after a switch, untimed
      CK(cudaEventRecord(e0, c->stream));
      for (int s = 0; s < n_steps; s++) CK(cudaGraphLaunch(c->gexec, c->stream));
      CK(cudaEventRecord(e1, c->stream));
      CK(cudaEventSynchronize(e1));
      float t;
      CK(cudaEventElapsedTime(&t, e0, e1));
      c->stages += 2 * (n_steps + 1);
      if (t < best_g) {
        best_g = t;
        shapes[3] = v;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->shape[3] = shapes[3];
    drop_graph(c);
  }
  return check_status(c);
}

int gks2l_alu_peaks(gks2l_ctx *c, double tflops[2]) {
  if (!c || !tflops) return GKS2L_EINVAL;
  if (!c->bound) return GKS2L_ESTATE;
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int nb = sms * 8, nth = 256;
  // the stores are never taken (the sums cannot equal the sentinel); the
  // staging area is large enough for every thread all the same
  if ((size_t)nb * nth > 18 * (size_t)c->prep.nt) return GKS2L_ESPACE;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const int it32 = 20000, it64 = 2000;
  for (int rep = 0; rep < 2; rep++) {
    float ms32 = 0, ms64 = 0;
    CK(cudaEventRecord(e0, c->stream));
    k_fma_probe<float><<<nb, nth, 0, c->stream>>>((float *)c->d_stage, it32, 0.999f, 0.001f);
    CK(cudaEventRecord(e1, c->stream));
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(&ms32, e0, e1));
    CK(cudaEventRecord(e0, c->stream));
    k_fma_probe<double><<<nb, nth, 0, c->stream>>>(c->d_stage, it64, 0.999, 0.001);
    CK(cudaEventRecord(e1, c->stream));
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(&ms64, e0, e1));
    tflops[0] = 16.0 * it32 * (double)nb * nth / (ms32 * 1e-3) / 1e12;
    tflops[1] = 16.0 * it64 * (double)nb * nth / (ms64 * 1e-3) / 1e12;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return GKS2L_OK;
}

int gks2l_set_mlp(gks2l_ctx *c, const float *params, size_t n_floats) {
  if (!c || !params || n_floats != (size_t)MLP_NPARAM) return GKS2L_EINVAL;
  if (!c->bound) return GKS2L_ESTATE;
  if (!(c->par.indicator_threshold > 0.f && c->par.indicator_threshold < 1.f)) return GKS2L_EINVAL;
  for (size_t i = 0; i < n_floats; i++)
    if (!std::isfinite(params[i])) return GKS2L_EINVAL;
  if (!c->side) {
    CK(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
  }
  float *tmp = nullptr;
  CK(cudaMallocAsync((void **)&tmp, n_floats * sizeof(float), c->stream));
  CK(cudaMemcpyAsync(tmp, params, n_floats * sizeof(float), cudaMemcpyHostToDevice, c->stream));
  const double t = c->par.indicator_threshold;
  k_mlp_pack<<<1, 256, 0, c->stream>>>(tmp, (float)std::log(t / (1.0 - t)), (MlpDev *)c->d.mlp);
  CK(cudaGetLastError());
  CK(cudaFreeAsync(tmp, c->stream));
  CK(cudaMemsetAsync(c->d.gate_mask, 0, (c->cs / TW) * sizeof(unsigned), c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->has_mlp = true;
  drop_graph(c);   // the captured step carries the gate switch
  return GKS2L_OK;
}

int gks2l_harvest(gks2l_ctx *c, float tol, float *d_features, float *d_labels, float *d_logits) {
  if (!c || !d_features || !d_labels || !(tol >= 0.f)) return GKS2L_EINVAL;
  if (!c->bound || !c->has_state) return GKS2L_ESTATE;
  if (d_logits && !c->has_mlp) return GKS2L_ESTATE;
  Par p = make_par(c);
  p.harvest = 1;
  float *ldev = nullptr;
  const size_t nt = c->prep.nt;
  if (d_logits) {
    CK(cudaMallocAsync((void **)&ldev, nt * sizeof(float), c->stream));
    p.logit_out = ldev;
  }
  // reconstruct the current state of every instance; the labels come from
  // the plain nonlinear weights, and the gate (if its logits are asked for)
  // runs on the same right-hand sides
  p.all_active = 1;
  p.use_gate = 0;
  const bool f32 = c->par.precision == GKS2L_FP32;
  if (d_logits) {
    if (f32) launch_gate<float>(c, p, c->stream);
    else launch_gate<double>(c, p, c->stream);
  }
  p.logit_out = nullptr;
  if (f32) {
    launch_recon<float>(c, p);
    k_harvest<float><<<blocks(nt, 128), 128, 0, c->stream>>>(c->d, c->d_perm, tol, ldev, d_features, d_labels,
                                                             d_logits);
  } else {
    launch_recon<double>(c, p);
    k_harvest<double><<<blocks(nt, 128), 128, 0, c->stream>>>(c->d, c->d_perm, tol, ldev, d_features, d_labels,
                                                              d_logits);
  }
  CK(cudaGetLastError());
  if (ldev) CK(cudaFreeAsync(ldev, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return GKS2L_OK;
}

const char *gks2l_error_string(int code) {
  switch (code) {
    case GKS2L_OK: return "ok";
    case GKS2L_EINVAL: return "invalid argument";
    case GKS2L_EMESH: return "mesh not usable";
    case GKS2L_ECUDA: return "CUDA runtime error";
    case GKS2L_ESTATE: return "call out of order";
    case GKS2L_ENEGDEPTH: return "non-positive depth";
    case GKS2L_ENONFINITE: return "non-finite value";
    case GKS2L_ESPACE: return "workspace too small";
    case GKS2L_ENOTIMPL: return "not implemented";
    case GKS2L_ETOOBIG: return "size beyond the fixed maximum of this entry point";
    case GKS2L_ETIMEOUT: return "a bounded device wait gave up";
    default: return "unknown status";
  }
}

void gks2l_destroy(gks2l_ctx *c) {
  if (!c) return;
  drop_graph(c);
  for (int b = 0; b < 2; b++) {
    if (c->io_in[b]) cudaFree(c->io_in[b]);
    if (c->io_out[b]) cudaFree(c->io_out[b]);
    for (cudaEvent_t e : {c->ev_in_ready[b], c->ev_in_free[b], c->ev_out_ready[b], c->ev_out_free[b]})
      if (e) cudaEventDestroy(e);
  }
  if (c->d_status_any) cudaFree(c->d_status_any);
  if (c->io_h2d) cudaStreamDestroy(c->io_h2d);
  if (c->io_d2h) cudaStreamDestroy(c->io_d2h);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  delete c;
}

}  // extern "C"
