// Per-thread work of one S2O4 stage of the compact two-layer GKS
// (arXiv 2306.04467), shared by the CUDA kernels in gks2l.cu. Each function
// handles one unit of work (a cell-variable, an edge Gauss point of one layer,
// or a cell) and is written as plain host/device code so the arithmetic of a
// unit does not depend on the launch shape.
//
// Deviation form. Every instance carries two FP64 reference values, R2 (a
// depth of the upper layer) and R1 (a water level eta1 = h1 + B of the lower
// layer): the area-weighted means of the state when it was set, rounded to
// 2^-32. The kernels read and write only deviations from them, of type R
// (double in the FP64 form, float in the FP32 form): the cell mirrors
// dq = (h2 - R2, h2U2, h2V2, eta1 - R1, h1U1, h1V1) and gradients
// dg = grad(h2, h2U2, h2V2, h1, h1U1, h1V1), the state's own gradients (so a
// state read out and set again is the same bit for bit); the reconstruction
// sees grad eta1 = grad h1 + grad B of each cell. At rest (eta1 and h2 constant,
// Sec. 3.2) every deviation vanishes, so the well-balanced cancellation
// between the interface flux and the cell sources holds in any precision: the
// reference pressure G (R1 - B)^2 / 2 of the lower layer is integrated around
// the cell exactly (B is linear, 2-point Gauss is exact) and combined with the
// bottom source analytically, leaving -G (eta1_j - R1) grad B_j. FP64 is kept
// for the cell averages, the mass fluxes and the state update, which keeps
// each layer's mass exactly conserved.
#pragma once
#include <cmath>
#include <cstdint>
#include <cstring>

#ifndef __CUDACC__
#define __host__
#define __device__
#define __forceinline__ inline
#endif

namespace gks2l {

#ifndef __CUDACC__
using std::isfinite;
#endif

constexpr int NV = 6;        // h2, h2U2, h2V2, h1 (as eta1 = h1 + B), h1U1, h1V1
constexpr int NSLOT = 9;
constexpr int NCOL = 17;
constexpr int NCOEF = 10;    // per variable: c0 (value offset) + 9 Taylor coefficients
// Side record of one cell for one layer: three slots of 12 values, one per
// variable of the layer (level, x- and y-discharge), each the 10 deviation
// coefficients, the cell-average deviation, then a constant: 1/h_s in slot 0,
// the bottom slope in slots 1-2 (lower layer; zero in the upper). An edge
// point reads its layer's record and slot 0 (the level) of the other layer's.
// 16-byte aligned, read with vector loads.
constexpr int NREC = 36;

// Device view of the workspace. R-typed arrays are stored as void* and cast.
struct Dev {
  int nt, ne, ninst;
  int cs;                   // stride of per-cell arrays (nt rounded up to 32)
  // per cell
  const int *inst;
  const double *area, *hs, *dX;
  const void *hsR, *ihsR;   // sqrt|Omega| and its inverse, type R
  const void *epsA;         // weno_eps * |Omega|, type R
  const void *bgR;          // [2][cell] grad B, type R
  const double *bmean, *bgx, *bgy;
  const int *st_cell;
  const int8_t *st_xf;
  const void *ops;          // per tile of 32 cells: the reconstruction's operator rows
  const void *plane;        // [(f*2+d)][cell] plane operator, type R
  const int *cedge;         // [f][cell]: edge id, or ~edge when the cell is the R side
  const double *fsl;        // [f][cell]: sign * |Gamma| / |Omega| (double, mass sums)
  const void *fslR;         // the same, type R (the other residuals)
  const int *inst_first;
  double *avg;              // state averages [v][cell] (FP64)
  void *dq, *dg;            // deviation mirrors [6][cell], gradients [12][cell], type R
  void *hrefc;              // R1 - B_j per cell, type R
  double *Wn, *Ln, *Ltn;    // stage snapshot (FP64; L and L_t rows of the layer depths only)
  void *incR;               // [4][cell] stage-1 part of the stage-2 momentum increment, type R
  void *srec;               // side records [layer][cell][NREC], type R (lower layer first)
  void *omg;                // omega_H / gamma_H of eta1 [0] and h2 [1], type R
  const void *mlp;          // gate network, packed image (MlpDev)
  unsigned *gate_mask;      // per tile of 32 cells: bit i = cell i takes the linear weights
  unsigned *gate_next;      // the gate's mask for the next reconstruction (k_update copies it over)
  // positivity option (not in the paper): per layer (0 lower, 1 upper) and
  // cell, whether the edge states' velocities are bounded, and the cell's
  // average depth
  unsigned char *pos_flag;  // [2][cs]
  void *pos_hbar;           // [2][cs], type R
                            // (written by one reconstruction for the next)
  float *wdev;              // [6][cell] max_k |omega_k / gamma_k - 1| (harvesting)
  // per edge
  const int *eL, *eR;
  const int8_t *exf;
  const void *en;           // [2][edge] unit normal from L to R, type R
  const double *eb0, *eb1;  // B at the two Gauss points
  const void *exiL, *exiR;  // [4][edge] Gauss points in each side's scaled frame, type R
  void *hrefe;              // [2][edge] R1 - B at the Gauss points, type R
  void *hc;                 // [2][edge] edge-centre blended level deviations, type R
  int *wl;                  // [2 * edge] (edge << 1 | layer) units left to the deferred edge pass
  int *wl_count;            // their number (zeroed before each fused edge launch)
  void *eF, *eFt, *eWt, *eWn;  // [6][edge] Gauss-point sums (weights 1/2), deviations, type R
  void *eO;                 // [side][layer][edge] each side's own level deviation, mean over
                            // the two Gauss points (the interlayer source's point values)
  double *eFm, *eFtm;       // [2][edge] the depth components of F, F_t (h2 first, then eta1) in
                            // FP64, converted once per edge for the cells' FP64 mass sums
  // per instance
  double *ref;              // [inst*2]: R2, R1
  void *refR;               // the same, type R
  double *dt, *t;
  void *dtR;                // dt, type R
  unsigned long long *dtbits;
  double *mass;             // [inst*2 + layer]
  int *status;
  unsigned long long *gate_count;
  const double *xf;         // [code*4] 2x2 linear parts of image transforms
};

struct Par {
  double g, chi, cfl, eps, eps_num, gam_hi, weno_eps;
  float gf, chif, epsf, eps_numf, gam_hif;   // the same in single precision
  int use_gate;                              // learned gate active
  float *logit_out;                          // gate logits per cell (device order), or null
  int all_active;                            // reconstruct every instance (harvesting)
  int harvest;                               // record the weights' departure from linear
  int staging_polls;                         // > 0: operator staging polls at most this many - 1 times
  double pos_floor;                          // positivity option (not in the paper): 0 = off
};

// a parameter in the form's precision
template <typename R> __host__ __device__ __forceinline__ R pv(double d, float f);
template <> __host__ __device__ __forceinline__ double pv<double>(double d, float) { return d; }
template <> __host__ __device__ __forceinline__ float pv<float>(double, float f) { return f; }

// erf(x) given ex = e^{-x^2}, which the caller has formed already: in FP64
// the library erf; in FP32 the rational approximation 7.1.26 of Abramowitz
// and Stegun (Handbook of Mathematical Functions, after Hastings),
// erf(|x|) = 1 - P(t) e^{-x^2}, P(t) = a1 t + ... + a5 t^5, t = 1/(1 + p|x|),
// absolute error at most 1.5e-7, with P re-expanded about t = 1 in
// s = 1 - t = p|x| t: P = b0 + b1 s + ... + b5 s^5, b_m = (-1)^m sum_k
// C(k, m) a_k, and b0 (= sum a_k = 1 - 1e-9) taken as 1, a change far inside
// that bound. Then erf(|x|) = (1 - e^{-x^2}) - e^{-x^2} s (b1 + ... + b5 s^4)
// has no cancellation at small |x|: it is exact at zero and proportional to x
// for tiny x (relative error 6e-6, the approximation's own slope), so the tiny
// velocities of a state near rest keep their size in the half-space moments'
// erf terms, which enter the deviation h-bar - h_b directly.
template <typename R> __host__ __device__ __forceinline__ R erf_ex(R x, R ex);
template <> __host__ __device__ __forceinline__ double erf_ex<double>(double x, double) { return erf(x); }
template <> __host__ __device__ __forceinline__ float erf_ex<float>(float x, float ex) {
  const float ax = x < 0.f ? -x : x;
  const float t = 1.f / (1.f + 0.3275911f * ax);
  const float s = 0.3275911f * ax * t;
  float q = -1.061405429f;
  q = q * s + 3.853875118f;
  q = q * s - 6.222859923f;
  q = q * s + 5.874886615f;
  q = q * s - 3.44449638f;
  const float e = (1.f - ex) - ex * s * q;
  return x < 0.f ? -e : e;
}
template <typename R> __host__ __device__ __forceinline__ R r_erfc(R x);
template <> __host__ __device__ __forceinline__ double r_erfc<double>(double x) { return erfc(x); }
template <> __host__ __device__ __forceinline__ float r_erfc<float>(float x) { return erfcf(x); }
template <typename R> __host__ __device__ __forceinline__ R r_exp(R x);
template <> __host__ __device__ __forceinline__ double r_exp<double>(double x) { return exp(x); }
// single precision on the device: the hardware exponential (a few ulp; the
// arguments here are O(1) Maxwellian exponents and -delta/tau)
template <> __host__ __device__ __forceinline__ float r_exp<float>(float x) {
#ifdef __CUDA_ARCH__
  return __expf(x);
#else
  return expf(x);
#endif
}
template <typename R> __host__ __device__ __forceinline__ R r_expm1(R x);
template <> __host__ __device__ __forceinline__ double r_expm1<double>(double x) { return expm1(x); }
template <> __host__ __device__ __forceinline__ float r_expm1<float>(float x) { return expm1f(x); }
template <typename R> __host__ __device__ __forceinline__ R r_sqrt(R x);
template <> __host__ __device__ __forceinline__ double r_sqrt<double>(double x) { return sqrt(x); }
template <> __host__ __device__ __forceinline__ float r_sqrt<float>(float x) { return sqrtf(x); }
template <typename R> __host__ __device__ __forceinline__ R r_abs(R x) { return x < 0 ? -x : x; }

// the bits of a double as a signed integer (> 0: positive, nonzero, and
// finite or NaN), and a finiteness test on them
__host__ __device__ __forceinline__ long long dbits(double x) {
#ifdef __CUDA_ARCH__
  return __double_as_longlong(x);
#else
  long long b;
  std::memcpy(&b, &x, sizeof b);
  return b;
#endif
}
__host__ __device__ __forceinline__ bool finite_bits(double x) { return ((dbits(x) >> 52) & 0x7ff) != 0x7ff; }

template <typename R>
__host__ __device__ __forceinline__ void monos(R x, R y, R m[10], R mx[10], R my[10]) {
  const R h = (R)0.5, s = (R)(1.0 / 6.0);
  R xx = x * x, yy = y * y, xy = x * y;
  const R one = (R)1, zero = (R)0;
  m[0] = one; m[1] = x; m[2] = y; m[3] = h * xx; m[4] = xy; m[5] = h * yy;
  m[6] = xx * x * s; m[7] = h * xx * y; m[8] = h * x * yy; m[9] = yy * y * s;
  mx[0] = zero; mx[1] = one; mx[2] = zero; mx[3] = x; mx[4] = y; mx[5] = zero;
  mx[6] = h * xx; mx[7] = xy; mx[8] = h * yy; mx[9] = zero;
  my[0] = zero; my[1] = zero; my[2] = one; my[3] = zero; my[4] = x; my[5] = y;
  my[6] = zero; my[7] = h * xx; my[8] = xy; my[9] = h * yy;
}

template <typename R>
__host__ __device__ __forceinline__ void rot2(const double *M, R v[2]) {
  R a = v[0], b = v[1];
  v[0] = (R)M[0] * a + (R)M[1] * b;
  v[1] = (R)M[2] * a + (R)M[3] * b;
}

// ------------------------------------------------------------------ cell data
// Deviation of reconstructed variable v of cell c seen through transform xf.
template <typename R>
__host__ __device__ __forceinline__ R img_dq(const Dev &d, int v, int c, int xf) {
  const int N = d.cs;
  const R *dq = (const R *)d.dq;
  if (v == 0 || v == 3 || xf == 0) return dq[v * N + c];
  int b = v < 3 ? 1 : 4;
  R m[2] = {dq[b * N + c], dq[(b + 1) * N + c]};
  rot2<R>(d.xf + 4 * xf, m);
  return m[v - b];
}
// gradient of reconstructed variable v of cell c seen through transform xf
// (for v = 3 the water level's: the stored grad h1 plus the cell's grad B)
template <typename R>
__host__ __device__ __forceinline__ void img_dg(const Dev &d, int v, int c, int xf, R g[2]) {
  const int N = d.cs;
  const R *G = (const R *)d.dg;
  if (v == 0 || v == 3 || xf == 0) {
    g[0] = G[(2 * v) * N + c];
    g[1] = G[(2 * v + 1) * N + c];
    if (v == 3) {
      g[0] += ((const R *)d.bgR)[c];
      g[1] += ((const R *)d.bgR)[N + c];
    }
    if (xf != 0) rot2<R>(d.xf + 4 * xf, g);
    return;
  }
  const double *M = d.xf + 4 * xf;
  // discharge gradient tensor T_ik = d m_i / d x_k -> M T M^T, row v - b
  int b = v < 3 ? 1 : 4;
  int row = v - b;
  R T[2][2] = {{G[(2 * b) * N + c], G[(2 * b + 1) * N + c]}, {G[(2 * b + 2) * N + c], G[(2 * b + 3) * N + c]}};
  for (int k = 0; k < 2; k++) {
    R s = 0;
    for (int a = 0; a < 2; a++)
      for (int b2 = 0; b2 < 2; b2++) s += (R)M[2 * row + a] * T[a][b2] * (R)M[2 * k + b2];
    g[k] = s;
  }
}

// --------------------------------------------------- compact reconstruction
// Operator rows of one cell: element k of row r is at base[r * stride + idx]
// (a tile staged in shared memory: stride = tile width, idx = cell in the tile).
template <typename R> struct CellOps {
  const R *lsq, *p1, *bq, *mm;
  const int *st;
  const int8_t *sx;
  int stride, idx;
};

// One cell and one variable: P3 least squares (Eq. Recons-system), three P1
// candidates on {cell, face neighbour}, smoothness indicators and WENO-Z
// weights, combined polynomial written as deviations in the Taylor basis.
// Three steps: gather the right-hand side, solve the P3 fit, then combine
// (where the troubled-cell gate can choose the linear weights).

// right-hand side: stencil average differences, then h-scaled gradients of
// the cell and its three face neighbours
template <typename R>
__host__ __device__ inline void recon_gather(const Dev &d, const CellOps<R> &o, int j, int v, R rhs[NCOL]) {
  const int N = d.cs, S = o.stride, I = o.idx;
  const R q0 = ((const R *)d.dq)[v * N + j];
  const R hs = ((const R *)d.hsR)[j];
  for (int s = 0; s < NSLOT; s++) {
    int c = o.st[s * S + I];
    rhs[s] = c >= 0 ? img_dq<R>(d, v, c, o.sx[s * S + I]) - q0 : (R)0;
  }
  R g[2];
  img_dg<R>(d, v, j, 0, g);
  rhs[9] = hs * g[0];
  rhs[10] = hs * g[1];
  for (int f = 0; f < 3; f++) {
    img_dg<R>(d, v, o.st[f * S + I], o.sx[f * S + I], g);
    rhs[11 + 2 * f] = hs * g[0];
    rhs[12 + 2 * f] = hs * g[1];
  }
}

// P3 least-squares coefficients a = M rhs
template <typename R>
__host__ __device__ inline void recon_p3(const CellOps<R> &o, const R rhs[NCOL], R a[9]) {
  const int S = o.stride, I = o.idx;
  for (int r = 0; r < 9; r++) {
    R s = 0;
    for (int c = 0; c < NCOL; c++) s += o.lsq[(r * NCOL + c) * S + I] * rhs[c];
    a[r] = s;
  }
}

// The result goes to the cell's side records: straight to global memory, or,
// with `stage` set, to a block's staging tile [layer][cell in tile][NREC]
// (o.stride cells per layer) that the block then writes out with 16-byte
// stores.
template <typename R>
__host__ __device__ inline void recon_finish(const Dev &d, const Par &p, const CellOps<R> &o, int j, int v,
                                             const R rhs[NCOL], const R a[9], bool linear, R *stage = nullptr) {
  const int N = d.cs, S = o.stride, I = o.idx;
  const R q0 = ((const R *)d.dq)[v * N + j];
  const R gh = pv<R>(p.gam_hi, p.gam_hif), gl = ((R)1 - gh) * (R)(1.0 / 3.0);
  R fac = 1, wf[3] = {gl, gl, gl}, b[3][2] = {{0, 0}, {0, 0}, {0, 0}};
  if (!linear) {
    R beta[4];
    for (int f = 0; f < 3; f++) {
      R r5[5] = {rhs[f], rhs[9], rhs[10], rhs[11 + 2 * f], rhs[12 + 2 * f]};
      for (int k = 0; k < 2; k++) {
        R s = 0;
        for (int c = 0; c < 5; c++) s += o.p1[((f * 2 + k) * 5 + c) * S + I] * r5[c];
        b[f][k] = s;
      }
      beta[1 + f] = b[f][0] * b[f][0] + b[f][1] * b[f][1];
    }
    R bh = 0;
    int idx = 0;
    for (int k = 0; k < 9; k++)
      for (int l = k; l < 9; l++) bh += o.bq[(idx++) * S + I] * a[k] * a[l];
    beta[0] = bh;
    R tz = (r_abs<R>(bh - beta[1]) + r_abs<R>(bh - beta[2]) + r_abs<R>(bh - beta[3])) * (R)(1.0 / 3.0);
    // the variable's value (reference + deviation) scales the regulariser
    R Q0 = q0;
    const R *refR = (const R *)d.refR;
    if (v == 0) Q0 += refR[2 * d.inst[j]];
    if (v == 3) Q0 += refR[2 * d.inst[j] + 1];
    R eps = ((const R *)d.epsA)[j] * (1 + Q0 * Q0);
    R w[4], ws = 0;
    const R gam[4] = {gh, gl, gl, gl};
    for (int k = 0; k < 4; k++) {
      R r = tz / (beta[k] + eps);
      w[k] = gam[k] * (1 + r * r);
      ws += w[k];
    }
    R iw = 1 / ws;
    fac = w[0] * iw / gh;
    for (int f = 0; f < 3; f++) wf[f] = w[1 + f] * iw;
    if (p.harvest) {
      R dv = r_abs<R>(fac - 1);
      for (int f = 0; f < 3; f++) {
        R df = r_abs<R>(wf[f] / gl - 1);
        dv = df > dv ? df : dv;
      }
      d.wdev[v * N + j] = (float)dv;
    }
  } else if (p.harvest) {
    d.wdev[v * N + j] = 0.f;
  }
  // R = (w_H / g_H)(P3 - sum g_m P1_m) + sum w_m P1_m
  R r[10];
  for (int k = 1; k < 10; k++) r[k] = fac * a[k - 1];
  for (int f = 0; f < 3; f++) {
    R cf = wf[f] - fac * gl;
    r[1] += cf * b[f][0];
    r[2] += cf * b[f][1];
  }
  R c0 = 0;
  for (int k = 3; k < 10; k++) c0 -= r[k] * o.mm[(k - 3) * S + I];
  r[0] = c0;
  // the layer's side record (vars 3,4,5 -> lower, 0,1,2 -> upper), and the
  // other layer's record for the level variables 0 and 3
  R *rec = stage ? stage : (R *)d.srec;
  const size_t ncell = stage ? (size_t)S : (size_t)N, cell = stage ? (size_t)I : (size_t)j;
  const int rs = NREC;
  R *p0 = rec + ((size_t)(v >= 3 ? 0 : 1) * ncell + cell) * rs + (v % 3) * 12;
  for (int k = 0; k < 10; k++) p0[k] = r[k];
  p0[10] = q0;
  if (v == 3) ((R *)d.omg)[j] = fac;
  if (v == 0) ((R *)d.omg)[N + j] = fac;
}

// ------------------------------------------------- evaluation at an edge point
// Edge-point side data for layer ell (0: lower, reconstructed eta1; 1: upper),
// all deviations of type R.
template <typename R> struct SideVals {
  R d;            // level deviation at the point (eta1 - R1 or h2 - R2)
  R h;            // depth at the point (href + d)
  R mx, my;       // discharge
  R gh[2];        // gradient of the depth
  R glev[2];      // gradient of the level variable
  R gm[2][2];     // discharge gradient tensor d m_i / d x_k
  R goth[2];      // gradient of the other layer's level variable
};

// cell c's reconstruction at scaled point (x, y), seen through transform xf;
// href is the depth of the reference level at the point
// n consecutive values of a side record (n a multiple of 4)
template <typename R, int n> __host__ __device__ __forceinline__ void load_rec(const R *p, R *w) {
  for (int k = 0; k < n; k++) w[k] = p[k];
}
#ifdef __CUDACC__
template <> __device__ __forceinline__ void load_rec<float, NREC>(const float *p, float *w) {
  const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
  for (int k = 0; k < NREC / 4; k++) {
    float4 t = q[k];
    w[4 * k] = t.x; w[4 * k + 1] = t.y; w[4 * k + 2] = t.z; w[4 * k + 3] = t.w;
  }
}
template <> __device__ __forceinline__ void load_rec<float, 12>(const float *p, float *w) {
  const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
  for (int k = 0; k < 3; k++) {
    float4 t = q[k];
    w[4 * k] = t.x; w[4 * k + 1] = t.y; w[4 * k + 2] = t.z; w[4 * k + 3] = t.w;
  }
}
template <> __device__ __forceinline__ void load_rec<double, NREC>(const double *p, double *w) {
  const double2 *q = reinterpret_cast<const double2 *>(p);
#pragma unroll
  for (int k = 0; k < NREC / 2; k++) {
    double2 t = q[k];
    w[2 * k] = t.x; w[2 * k + 1] = t.y;
  }
}
template <> __device__ __forceinline__ void load_rec<double, 12>(const double *p, double *w) {
  const double2 *q = reinterpret_cast<const double2 *>(p);
#pragma unroll
  for (int k = 0; k < 6; k++) {
    double2 t = q[k];
    w[2 * k] = t.x; w[2 * k + 1] = t.y;
  }
}
#endif

// Operations rounded as written, whatever the compiler does with the code
// around them: where two kernels must form the same value bit for bit.
template <typename R> struct Rn;
template <> struct Rn<float> {
#ifdef __CUDA_ARCH__
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
  static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
  static __device__ __forceinline__ float rcp(float a) { return __frcp_rn(a); }
#else
  static float mul(float a, float b) { return a * b; }
  static float add(float a, float b) { return a + b; }
  static float sub(float a, float b) { return a - b; }
  static float fma(float a, float b, float c) { return std::fma(a, b, c); }
  static float rcp(float a) { return 1.0f / a; }
#endif
};
template <> struct Rn<double> {
#ifdef __CUDA_ARCH__
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
  static __device__ __forceinline__ double rcp(double a) { return __drcp_rn(a); }
#else
  static double mul(double a, double b) { return a * b; }
  static double add(double a, double b) { return a + b; }
  static double sub(double a, double b) { return a - b; }
  static double fma(double a, double b, double c) { return std::fma(a, b, c); }
  static double rcp(double a) { return 1.0 / a; }
#endif
};

// gradient (scaled by ih) of the level polynomial cf at a point's monomial
// derivatives, explicitly rounded: the edge kernels take the other layer's
// level gradient from the lane that formed it as its own, the deferred edge
// pass forms it again, and both get the same bits
template <typename R>
__host__ __device__ __forceinline__ void level_grad(const R *cf, const R mx[10], const R my[10], R ih, R g[2]) {
  using O = Rn<R>;
  R ax = cf[1], ay = cf[2];
  for (int k : {3, 4, 6, 7, 8}) ax = O::fma(cf[k], mx[k], ax);
  for (int k : {4, 5, 7, 8, 9}) ay = O::fma(cf[k], my[k], ay);
  g[0] = O::mul(ax, ih);
  g[1] = O::mul(ay, ih);
}
// 2x2 rotation, explicitly rounded (for the level gradients above)
template <typename R>
__host__ __device__ __forceinline__ void rot2_rn(const double *M, R v[2]) {
  using O = Rn<R>;
  const R a = v[0], b = v[1];
  v[0] = O::fma((R)M[1], b, O::mul((R)M[0], a));
  v[1] = O::fma((R)M[3], b, O::mul((R)M[2], a));
}

// One side of an edge point: cell c's reconstruction of layer ell at scaled
// point (x, y), seen through transform xf; href is the depth of the
// reference level at the point. OTHER: also form the gradient of the other
// layer's level from its record (otherwise the caller takes it from the lane
// that forms it as its own).
template <typename R, bool OTHER = true>
__host__ __device__ inline void side_vals(const Dev &d, int ell, int c, int xf, R x, R y, R href, SideVals<R> &s) {
  const int N = d.cs;
  R w[NREC];
  load_rec<R, NREC>((const R *)d.srec + ((size_t)ell * N + c) * NREC, w);
  R m[10], mx[10], my[10];
  monos<R>(x, y, m, mx, my);
  const R ih = w[11];
  R dev[3], gx[3], gy[3];
  for (int i = 0; i < 3; i++) {
    const R *cf = w + 12 * i;
    R a = cf[0] * m[0];
    for (int k = 1; k < 10; k++) a += cf[k] * m[k];
    dev[i] = a;
    if (i == 0) {
      R g[2];
      level_grad<R>(cf, mx, my, ih, g);
      gx[0] = g[0];
      gy[0] = g[1];
    } else {
      R ax = cf[1] * mx[1], ay = cf[2] * my[2];
      for (int k : {3, 4, 6, 7, 8}) ax += cf[k] * mx[k];
      for (int k : {4, 5, 7, 8, 9}) ay += cf[k] * my[k];
      gx[i] = ax * ih;
      gy[i] = ay * ih;
    }
  }
  s.goth[0] = s.goth[1] = 0;
  if (OTHER) {
    R wo[12];
    load_rec<R, 12>((const R *)d.srec + ((size_t)(1 - ell) * N + c) * NREC, wo);
    level_grad<R>(wo, mx, my, ih, s.goth);
  }
  s.d = w[10] + dev[0];
  s.h = href + s.d;
  s.mx = w[22] + dev[1];
  s.my = w[34] + dev[2];
  s.glev[0] = gx[0]; s.glev[1] = gy[0];
  s.gm[0][0] = gx[1]; s.gm[0][1] = gy[1];
  s.gm[1][0] = gx[2]; s.gm[1][1] = gy[2];
  R gb[2] = {0, 0};
  if (ell == 0) { gb[0] = w[23]; gb[1] = w[35]; }
  if (xf != 0) {
    const double *M = d.xf + 4 * xf;
    R mv[2] = {s.mx, s.my};
    rot2<R>(M, mv);
    s.mx = mv[0]; s.my = mv[1];
    rot2_rn<R>(M, s.glev);
    if (OTHER) rot2_rn<R>(M, s.goth);
    rot2<R>(M, gb);
    R G2[2][2] = {{s.gm[0][0], s.gm[0][1]}, {s.gm[1][0], s.gm[1][1]}};
    for (int i2 = 0; i2 < 2; i2++)
      for (int k = 0; k < 2; k++) {
        R acc = (R)M[2 * i2] * G2[0][0] * (R)M[2 * k] + (R)M[2 * i2] * G2[0][1] * (R)M[2 * k + 1];
        acc += (R)M[2 * i2 + 1] * G2[1][0] * (R)M[2 * k];
        acc += (R)M[2 * i2 + 1] * G2[1][1] * (R)M[2 * k + 1];
        s.gm[i2][k] = acc;
      }
  }
  s.gh[0] = s.glev[0] - gb[0];   // depth = level - B for the lower layer
  s.gh[1] = s.glev[1] - gb[1];
}

// the level deviation and the discharges at scaled point (x, y) from a
// loaded side record
template <typename R>
__host__ __device__ __forceinline__ void rec_values(const R *w, R x, R y, R v[3]) {
  const R hh = (R)0.5, s6 = (R)(1.0 / 6.0);
  const R xx = x * x, yy = y * y, xy = x * y;
  const R m[10] = {(R)1, x, y, hh * xx, xy, hh * yy, xx * x * s6, hh * xx * y, hh * x * yy, yy * y * s6};
  for (int i = 0; i < 3; i++) {
    R a = w[12 * i] * m[0];
    for (int k = 1; k < 10; k++) a += w[12 * i + k] * m[k];
    v[i] = w[12 * i + 10] + a;
  }
}

// depth of the reference level at Gauss point q of edge e for layer ell
template <typename R>
__host__ __device__ __forceinline__ R ref_depth(const Dev &d, int ell, int e, int q) {
  if (ell == 0) return ((const R *)d.hrefe)[q * d.ne + e];
  return ((const R *)d.refR)[2 * d.inst[d.eL[e]]];
}

// ------------------------------------------------ gas-kinetic interface solution
template <typename R> struct Kern {
  R gu, gv, puu, puv, pvv, bu, bv;
};

// Central moments mu_k = <c^k> (k = 0..5, c = u - U) of the normalised 1-D
// Maxwellian over the half line sgn*u > 0, from E = e^{-lam U^2}/(2 sqrt(pi lam))
// (formed by the caller); e0 = mu_0 - 1/2.
template <typename R>
__host__ __device__ __forceinline__ void half_moments_E(R U, R lam, R sgn, R E, R ex, R mu[6], R &e0) {
  const R th = (R)0.5 / lam;
  e0 = sgn * (R)0.5 * erf_ex<R>(r_sqrt<R>(lam) * U, ex);   // ex = e^{-lam U^2}
  mu[0] = (R)0.5 + e0;
  mu[1] = sgn * E;
  R pw = -sgn * U * E;
  mu[2] = th * mu[0] + pw;
  pw *= -U;
  mu[3] = 2 * th * mu[1] + pw;
  pw *= -U;
  mu[4] = 3 * th * mu[2] + pw;
  pw *= -U;
  mu[5] = 4 * th * mu[3] + pw;
}

// both half lines of one Maxwellian (sgn = +1 into mp, -1 into mm), sharing
// its error function and exponential
template <typename R>
__host__ __device__ __forceinline__ void half_moments_pm(R U, R lam, R mp[6], R mm[6]) {
  const R th = (R)0.5 / lam;
  const R ex = r_exp<R>(-lam * U * U);
  const R e0 = (R)0.5 * erf_ex<R>(r_sqrt<R>(lam) * U, ex);
  const R E = ex * (R)0.5 / r_sqrt<R>((R)3.14159265358979323846 * lam);
  for (int sg = 0; sg < 2; sg++) {
    const R sgn = sg == 0 ? (R)1 : (R)-1;
    R *mu = sg == 0 ? mp : mm;
    mu[0] = (R)0.5 + sgn * e0;
    mu[1] = sgn * E;
    R pw = -sgn * U * E;
    mu[2] = th * mu[0] + pw;
    pw *= -U;
    mu[3] = 2 * th * mu[1] + pw;
    pw *= -U;
    mu[4] = 3 * th * mu[2] + pw;
    pw *= -U;
    mu[5] = 4 * th * mu[3] + pw;
  }
}

// Slope + force kernel on a Maxwellian base (h, U, V, lam), written as a
// polynomial in c = u - U: the exact derivative of ln g along n and t, plus
// the force term, whose cubic part combines into (lam/h) |c|^2 (D . c) with
// D = grad h - grad Phi / G (local frame).
template <typename R>
__host__ __device__ __forceinline__ Kern<R> make_kern(R h, R U, R V, R lam, const R dn[3], const R dt[3],
                                                      const R D[2]) {
  Kern<R> K;
  R ih = 1 / h;
  R aun = (dn[1] - U * dn[0]) * ih, avn = (dn[2] - V * dn[0]) * ih;
  R aut = (dt[1] - U * dt[0]) * ih, avt = (dt[2] - V * dt[0]) * ih;
  R al = lam * ih * (dn[0] * U + dt[0] * V);
  R tl = 2 * lam;
  K.gu = tl * (aun * U + aut * V);
  K.gv = tl * (avn * U + avt * V);
  K.puu = al + tl * aun;
  K.pvv = al + tl * avt;
  K.puv = tl * (avn + aut);
  K.bu = lam * ih * D[0];
  K.bv = lam * ih * D[1];
  return K;
}

// moments of the kernel with weights (1, u, v) and (u, u^2, uv), per unit density
template <typename R>
__host__ __device__ __forceinline__ void kern_moments(const Kern<R> &K, const R mu[6], R th, R U, R V, R out[6]) {
  const R n2 = th, n4 = 3 * th * th;
  R T00 = K.gu * mu[1] + K.puu * mu[2] + K.pvv * mu[0] * n2 + K.bu * (mu[3] + mu[1] * n2);
  R T10 = K.gu * mu[2] + K.puu * mu[3] + K.pvv * mu[1] * n2 + K.bu * (mu[4] + mu[2] * n2);
  R T20 = K.gu * mu[3] + K.puu * mu[4] + K.pvv * mu[2] * n2 + K.bu * (mu[5] + mu[3] * n2);
  R T01 = K.gv * mu[0] * n2 + K.puv * mu[1] * n2 + K.bv * (mu[2] * n2 + mu[0] * n4);
  R T11 = K.gv * mu[1] * n2 + K.puv * mu[2] * n2 + K.bv * (mu[3] * n2 + mu[1] * n4);
  out[0] = T00;
  out[1] = U * T00 + T10;
  out[2] = V * T00 + T01;
  out[3] = out[1];
  out[4] = U * U * T00 + 2 * U * T10 + T20;
  out[5] = U * V * T00 + V * T10 + U * T01 + T11;
}

// time integrals over [0, delta] of C1..C5, from e = exp(-delta/tau) and
// em = 1 - e
template <typename R>
__host__ __device__ __forceinline__ void time_ints_e(R tau, R delta, R e, R em, R q[5]) {
  q[0] = delta - tau * em;
  q[1] = -tau * delta * (1 + e) + 2 * tau * tau * em;
  q[2] = (R)0.5 * delta * delta - tau * delta + tau * tau * em;
  q[3] = tau * em;
  q[4] = tau * delta * e - tau * tau * em;
}
// the same over [0, delta] (qd) and [0, delta / 2] (qh); the full interval's
// exponentials follow from the half interval's: e = eh^2, 1 - e = emh (1 + eh)
template <typename R>
__host__ __device__ __forceinline__ void time_ints2(R tau, R delta, R qd[5], R qh[5]) {
  const R xh = (R)0.5 * delta / tau;
  const R emh = -r_expm1<R>(-xh), eh = r_exp<R>(-xh);
  time_ints_e<R>(tau, (R)0.5 * delta, eh, emh, qh);
  time_ints_e<R>(tau, delta, eh * eh, emh * (1 + eh), qd);
}

// One layer at one Gauss point, local frame (x along the normal from L to R).
// Depths h_l = href + dl, h_r = href + dr. Returns the value and time
// derivative at the stage start of the flux F and of the interface variables
// W (fit of the two time integrals over delta and delta/2), as deviations:
// the normal-momentum flux minus G href^2 / 2 and the depth minus href.
template <typename R>
__host__ __device__ inline void gks_layer(R href, R dl, R dr, R Ul, R Vl, R Ur, R Vr, const R dnl[3],
                                          const R dtl[3], const R Dl[2], const R dnr[3], const R dtr[3],
                                          const R Dr[2], R g, R tau, R delta, R F[3], R Ft[3], R W[3], R Wt[3]) {
  const R hlR = href + dl, hrR = href + dr;
  const R dlr = dl - dr;                          // h_l - h_r, exact at rest
  const R laml = 1 / (g * hlR), lamr = 1 / (g * hrR);
  const R thl = (R)0.5 * g * hlR, thr = (R)0.5 * g * hrR;
  // E = e^{-lam U^2} / (2 sqrt(pi lam)) = sqrt(G/(4 pi)) sqrt(h) e^{-lam U^2}
  // on each side: one exponential and one square root serve the half-space
  // moments and the depth-difference term below
  const R xl = r_exp<R>(-laml * Ul * Ul), xr = r_exp<R>(-lamr * Ur * Ur);
  const R sl = r_sqrt<R>(hlR), sr = r_sqrt<R>(hrR);
  const R cphi = r_sqrt<R>(g * (R)(0.25 / 3.14159265358979323846));
  const R El = cphi * sl * xl, Er = cphi * sr * xr;
  R mul[6], mur[6], e0l, e0r;
  half_moments_E<R>(Ul, laml, (R)1, El, xl, mul, e0l);
  half_moments_E<R>(Ur, lamr, (R)-1, Er, xr, mur, e0r);
  // W-bar: the t = 0 interface state; h_b = (h_l + h_r)/2, h-bar = h_b + hdev
  const R db = (R)0.5 * (dl + dr);                // h_b - href
  const R hb = href + db;
  const R hdev = hlR * e0l + hrR * e0r;
  // h_l E_l - h_r E_r with h E = sqrt(G/(4 pi)) h^{3/2} e^{-lam U^2}, written
  // through h_l - h_r so that it vanishes exactly for equal depths and velocities
  const R dphi = dlr * (hlR + sl * sr + hrR) / (sl + sr);
  const R ediff = cphi * (hlR * sl * (xl - xr) + dphi * xr);
  const R mbn = (hlR * Ul * mul[0] + hrR * Ur * mur[0]) + ediff;
  const R mbt = hlR * Vl * mul[0] + hrR * Vr * mur[0];
  const R hbR = hb + hdev;
  const R Ub = mbn / hbR, Vb = mbt / hbR;
  const R lamb = 1 / (g * hbR), thb = (R)0.5 * g * hbR;
  R mbp[6], mbm[6];
  half_moments_pm<R>(Ub, lamb, mbp, mbm);
  Kern<R> kbl = make_kern<R>(hbR, Ub, Vb, lamb, dnl, dtl, Dl);
  Kern<R> kbr = make_kern<R>(hbR, Ub, Vb, lamb, dnr, dtr, Dr);
  Kern<R> kl = make_kern<R>(hlR, Ul, Vl, laml, dnl, dtl, Dl);
  Kern<R> kr = make_kern<R>(hrR, Ur, Vr, lamr, dnr, dtr, Dr);
  R P[5][6], a[6], b[6];
  // C2: equilibrium slopes and force, two-sided
  kern_moments<R>(kbl, mbp, thb, Ub, Vb, a);
  kern_moments<R>(kbr, mbm, thb, Ub, Vb, b);
  for (int k = 0; k < 6; k++) P[1][k] = hbR * (a[k] + b[k]);
  // C3: A-bar from compatibility, d = time derivative of (h, hU, hV)
  const R dh = -P[1][0], dm = -P[1][1], dn = -P[1][2];
  P[2][0] = dh; P[2][1] = dm; P[2][2] = dn;
  P[2][3] = dm;
  P[2][4] = 2 * Ub * dm - Ub * Ub * dh + 2 * thb * dh;
  P[2][5] = Vb * dm + Ub * dn - Ub * Vb * dh;
  // C5: free transport of the initial slopes and force
  kern_moments<R>(kl, mul, thl, Ul, Vl, a);
  kern_moments<R>(kr, mur, thr, Ur, Vr, b);
  for (int k = 0; k < 6; k++) P[4][k] = hlR * a[k] + hrR * b[k];
  // C1 (full-space moments of g-bar) and C4 (g^l, g^r on their half spaces):
  // deviations from the bases h_b and G h_b^2 / 2
  P[0][0] = hdev; P[0][1] = mbn; P[0][2] = mbt;
  P[0][3] = mbn;
  P[0][4] = mbn * Ub + g * hb * hdev + (R)0.5 * g * hdev * hdev;
  P[0][5] = mbn * Vb;
  P[3][0] = hdev; P[3][1] = mbn; P[3][2] = mbt;
  P[3][3] = mbn;
  {
    const R m2l = thl * e0l - Ul * El, m2r = thr * e0r + Ur * Er;   // mu_2 - th/2 on each side
    P[3][4] = hlR * (Ul * Ul * mul[0] + 2 * Ul * mul[1] + m2l) + hrR * (Ur * Ur * mur[0] + 2 * Ur * mur[1] + m2r) +
              (R)0.125 * g * dlr * dlr;
  }
  P[3][5] = hlR * Vl * (Ul * mul[0] + mul[1]) + hrR * Vr * (Ur * mur[0] + mur[1]);
  // fitted value and derivative at the stage start
  R qd[5], qh[5];
  time_ints2<R>(tau, delta, qd, qh);
  R kv[5], kd[5];
  const R id = 1 / delta;
  for (int i = 0; i < 5; i++) {
    kv[i] = (4 * qh[i] - qd[i]) * id;
    kd[i] = 4 * (qd[i] - 2 * qh[i]) * id * id;
  }
  R f[3], ft[3], w[3], wt[3];
  for (int k = 0; k < 3; k++) {
    w[k] = kv[0] * P[0][k];
    wt[k] = kd[0] * P[0][k];
    f[k] = kv[0] * P[0][3 + k];
    ft[k] = kd[0] * P[0][3 + k];
  }
  for (int i = 1; i < 5; i++)
    for (int k = 0; k < 3; k++) {
      w[k] += kv[i] * P[i][k];
      wt[k] += kd[i] * P[i][k];
      f[k] += kv[i] * P[i][3 + k];
      ft[k] += kd[i] * P[i][3 + k];
    }
  // bases relative to the reference: h_b - href and G (h_b^2 - href^2) / 2
  W[0] = db + w[0];
  W[1] = w[1];
  W[2] = w[2];
  F[0] = f[0];
  F[1] = (R)0.5 * g * db * (hb + href) + f[1];
  F[2] = f[2];
  for (int k = 0; k < 3; k++) { Wt[k] = wt[k]; Ft[k] = ft[k]; }
}

// Blended level deviation at one point (Sec. 2.3): d^r + xi (d^l - d^r) with
// xi = erfc((U_n^l + U_n^r)/2)/2, U_n = (m . n) / h on each side. Written
// with explicitly rounded operations so that the interface kernel and the
// fused edge kernel, which both form it, get the same value whatever the
// compiler does with the code around it.
template <typename R>
__host__ __device__ __forceinline__ R blend_level(R dl, R hl, R mxl, R myl, R dr, R hr, R mxr, R myr, R n0, R n1) {
  using O = Rn<R>;
  const R ul = O::mul(O::fma(mxl, n0, O::mul(myl, n1)), O::rcp(hl));
  const R ur = O::mul(O::fma(mxr, n0, O::mul(myr, n1)), O::rcp(hr));
  const R xi = O::mul((R)0.5, r_erfc<R>(O::mul((R)0.5, O::add(ul, ur))));
  return O::fma(xi, O::sub(dl, dr), dr);
}

// ---------------------------------------------------- interface (iface) unit
// Blended level deviation of layer ell at edge e (Sec. 2.3), the mean over
// the two Gauss points of h-hat = xi h^l + (1 - xi) h^r with
// xi = erfc((U_n^l + U_n^r)/2)/2; the lower layer is blended as the water
// level eta1 (B is continuous). Each side's record is loaded once for both
// points.
template <typename R>
__host__ __device__ inline R iface_unit(const Dev &d, int e, int ell) {
  const int NE = d.ne, N = d.cs;
  const R *xl = (const R *)d.exiL, *xr = (const R *)d.exiR, *en = (const R *)d.en;
  const int cL = d.eL[e], cR = d.eR[e], xf = d.exf[e];
  R vl[2][3], vr[2][3];
  {
    R w[NREC];
    load_rec<R, NREC>((const R *)d.srec + ((size_t)ell * N + cL) * NREC, w);
    for (int q = 0; q < 2; q++) rec_values<R>(w, xl[(2 * q) * NE + e], xl[(2 * q + 1) * NE + e], vl[q]);
  }
  {
    R w[NREC];
    load_rec<R, NREC>((const R *)d.srec + ((size_t)ell * N + cR) * NREC, w);
    for (int q = 0; q < 2; q++) rec_values<R>(w, xr[(2 * q) * NE + e], xr[(2 * q + 1) * NE + e], vr[q]);
  }
  const R n0 = en[e], n1 = en[NE + e];
  R v[2];
  for (int q = 0; q < 2; q++) {
    R mr[2] = {vr[q][1], vr[q][2]};
    if (xf != 0) rot2<R>(d.xf + 4 * xf, mr);
    const R href = ref_depth<R>(d, ell, e, q);
    const R dl = vl[q][0], dr = vr[q][0];
    v[q] = blend_level<R>(dl, href + dl, vl[q][1], vl[q][2], dr, href + dr, mr[0], mr[1], n0, n1);
  }
  return Rn<R>::mul((R)0.5, Rn<R>::add(v[0], v[1]));
}

// plane gradient (Sec. 2.3) of the blended level `which` for cell c
template <typename R>
__host__ __device__ __forceinline__ void plane_grad(const Dev &d, int c, int which, R g[2]) {
  const int N = d.cs, NE = d.ne;
  const R *pl = (const R *)d.plane, *hc = (const R *)d.hc;
  g[0] = g[1] = 0;
  for (int f = 0; f < 3; f++) {
    int ce = d.cedge[f * N + c];
    int e = ce >= 0 ? ce : ~ce;
    R v = hc[which * NE + e];
    g[0] += pl[(f * 2) * N + c] * v;
    g[1] += pl[(f * 2 + 1) * N + c] * v;
  }
}

// ------------------------------------------------------------- edge unit
// Interface solution of layer ell at Gauss point q of edge e, global frame:
// out[0..2] = F, out[3..5] = F_t, out[6..8] = W, out[9..11] = W_t (deviations).
// Returns true when out was computed.
// FUSED (runs with the troubled-cell gate, where most cells take the linear
// weights): the unit also returns in *blend the point's blended level
// deviation of layer ell, h-hat - href = d^r + xi (d^l - d^r) with
// xi = erfc((U_n^l + U_n^r)/2)/2 (Sec. 2.3; the edge's blended level is the
// mean over its two points), and computes the solution only where the blend
// weight w of the other layer is 1, where the plane gradients, which need
// every blended level of both cells, carry no weight; elsewhere it returns
// false and the solution is left to a later pass (plain mode, plane
// gradients gathered).
// PAIRED (the edge kernels' thread layout, where the lane two over holds the
// same point and side for the other layer): the other layer's level
// gradient comes from that lane by a shuffle instead of from its record.
// POS (the positivity option, not in the paper): on a side whose cell's
// layer has point depths below half its average, the side velocity is
// bounded by the edge's two cells' average velocities of the layer.
template <typename R, bool FUSED = false, bool PAIRED = false, bool POS = false>
__host__ __device__ inline bool edge_unit(const Dev &d, const Par &p, int e, int ell, int q, int stage, R out[12],
                                          R *blend = nullptr, R *own = nullptr) {
  const int NE = d.ne;
  const R *xl = (const R *)d.exiL, *xr = (const R *)d.exiR, *en = (const R *)d.en;
  int cL = d.eL[e], cR = d.eR[e], xf = d.exf[e];
  const R dt = ((const R *)d.dtR)[d.inst[cL]];
  // both stages fit the value and time derivative at their start from the
  // time integrals over dt and dt/2 (the S2O4 construction repeated from the
  // intermediate state, reading R20)
  const R delta = dt;
  (void)stage;
  const R href = ref_depth<R>(d, ell, e, q);
  SideVals<R> s[2];
#ifdef __CUDA_ARCH__
  constexpr bool SH = PAIRED;
#else
  constexpr bool SH = false;
#endif
  side_vals<R, !SH>(d, ell, cL, 0, xl[(2 * q) * NE + e], xl[(2 * q + 1) * NE + e], href, s[0]);
  side_vals<R, !SH>(d, ell, cR, xf, xr[(2 * q) * NE + e], xr[(2 * q + 1) * NE + e], href, s[1]);
#ifdef __CUDA_ARCH__
  if (SH) {
    for (int sd = 0; sd < 2; sd++)
      for (int k = 0; k < 2; k++) s[sd].goth[k] = __shfl_xor_sync(0xffffffffu, s[sd].glev[k], 2);
  }
#endif
  // blended derivative of the other layer's level and the well-balance vector
  // D = grad h - grad Phi / G = grad(level) + c (w grad(other) + (1 - w) grad P1)
  const int oth = 1 - ell;  // hc / omg index of the other layer: 0 = eta1, 1 = h2
  const R *om = (const R *)d.omg;
  R w = om[oth * d.cs + cL] < om[oth * d.cs + cR] ? om[oth * d.cs + cL] : om[oth * d.cs + cR];
  w = w < (R)0 ? (R)0 : (w > (R)1 ? (R)1 : w);
  // the plane gradients enter with weight 1 - w (the fused mode computes
  // only units with w = 1)
  R pl[2][2] = {{0, 0}, {0, 0}};
  if (!FUSED) {
    plane_grad<R>(d, cL, oth, pl[0]);
    plane_grad<R>(d, cR, oth, pl[1]);
    if (xf != 0) rot2<R>(d.xf + 4 * xf, pl[1]);
  }
  const R cf = ell == 0 ? pv<R>(p.chi, p.chif) : (R)1;
  const R n0 = en[e], n1 = en[NE + e];
  R U[2], V[2], dn[2][3], dtt[2][3], D[2][2];
  for (int sd = 0; sd < 2; sd++) {
    const SideVals<R> &S = s[sd];
    R Dx = S.glev[0] + cf * (w * S.goth[0] + (1 - w) * pl[sd][0]);
    R Dy = S.glev[1] + cf * (w * S.goth[1] + (1 - w) * pl[sd][1]);
    D[sd][0] = Dx * n0 + Dy * n1;
    D[sd][1] = -Dx * n1 + Dy * n0;
    R ih = (R)1 / S.h;
    U[sd] = (S.mx * n0 + S.my * n1) * ih;
    V[sd] = (-S.mx * n1 + S.my * n0) * ih;
    // derivatives along n and t of (h, m_n, m_t)
    const R dir[2][2] = {{n0, n1}, {-n1, n0}};
    R *outv[2] = {dn[sd], dtt[sd]};
    for (int k = 0; k < 2; k++) {
      R ex = dir[k][0], ey = dir[k][1];
      R dhh = S.gh[0] * ex + S.gh[1] * ey;
      R dmx = S.gm[0][0] * ex + S.gm[0][1] * ey;
      R dmy = S.gm[1][0] * ex + S.gm[1][1] * ey;
      outv[k][0] = dhh;
      outv[k][1] = dmx * n0 + dmy * n1;
      outv[k][2] = -dmx * n1 + dmy * n0;
    }
  }
  if (POS) {
    const int N = d.cs, vm = ell == 0 ? 4 : 1;
    const bool bl = d.pos_flag[ell * N + cL] != 0, br = d.pos_flag[ell * N + cR] != 0;
    if (bl || br) {
      const R *hb = (const R *)d.pos_hbar;
      R un[2], ut[2];
      for (int sd = 0; sd < 2; sd++) {
        const int c = sd == 0 ? cL : cR, x = sd == 0 ? 0 : xf;
        const R mx = img_dq<R>(d, vm, c, x), my = img_dq<R>(d, vm + 1, c, x);
        const R ih = (R)1 / hb[ell * N + c];
        un[sd] = (mx * n0 + my * n1) * ih;
        ut[sd] = (-mx * n1 + my * n0) * ih;
      }
      const R ulo = un[0] < un[1] ? un[0] : un[1], uhi = un[0] < un[1] ? un[1] : un[0];
      const R tlo = ut[0] < ut[1] ? ut[0] : ut[1], thi = ut[0] < ut[1] ? ut[1] : ut[0];
      for (int sd = 0; sd < 2; sd++) {
        if (!(sd == 0 ? bl : br)) continue;
        U[sd] = U[sd] < ulo ? ulo : (U[sd] > uhi ? uhi : U[sd]);
        V[sd] = V[sd] < tlo ? tlo : (V[sd] > thi ? thi : V[sd]);
      }
    }
  }
  // each side's own level at the point: the interlayer source's values (R16)
  if (own) {
    own[0] = s[0].d;
    own[1] = s[1].d;
  }
  if (FUSED) {
    *blend = blend_level<R>(s[0].d, s[0].h, s[0].mx, s[0].my, s[1].d, s[1].h, s[1].mx, s[1].my, n0, n1);
    if (w < (R)1) return false;
  }
  // collision time (Sec. 4): tau = eps dt + eps_num |(hl^2 - hr^2)/(hl^2 + hr^2)| dt
  const R hl = s[0].h, hr = s[1].h;
  const R jump = r_abs<R>((s[0].d - s[1].d) * (hl + hr) / (hl * hl + hr * hr));
  const R tau = pv<R>(p.eps, p.epsf) * dt + pv<R>(p.eps_num, p.eps_numf) * jump * dt;
  R F[3], Ft[3], W[3], Wt[3];
  gks_layer<R>(href, s[0].d, s[1].d, U[0], V[0], U[1], V[1], dn[0], dtt[0], D[0], dn[1], dtt[1], D[1],
               pv<R>(p.g, p.gf), tau, delta, F, Ft, W, Wt);
  const R *src[4] = {F, Ft, W, Wt};
  for (int k = 0; k < 4; k++) {
    out[3 * k] = src[k][0];
    out[3 * k + 1] = src[k][1] * n0 - src[k][2] * n1;
    out[3 * k + 2] = src[k][1] * n1 + src[k][2] * n0;
  }
  return true;
}

// ------------------------------------------------------------- cell unit
// dX / U_max of a cell state w (Sec. 4: U_max the larger over the layers of
// |U| + sqrt(G h)) in the form's precision; the update kernel and the kernel
// that starts a newly set state both use it, so a restarted run takes the
// same steps as an uninterrupted one. FP32 form: the reciprocal in single
// precision (dt to ~1e-7 relative), sparing the FP64 pipe a double division.
template <typename R>
__host__ __device__ inline double cfl_ratio(const double w[NV], double dX, R G) {
  R um = 0;
  for (int l = 0; l < 2; l++) {
    R h = (R)w[3 * l], u = (R)w[3 * l + 1] / h, v = (R)w[3 * l + 2] / h;
    R sp = r_sqrt<R>(u * u + v * v) + r_sqrt<R>(G * h);
    um = sp > um ? sp : um;
  }
  if (sizeof(R) == 4) return dX * (double)((R)1 / um);
  return dX / (double)um;
}

// Flux and source residuals, S2O4 update (Eq. SWE-fully-discrete), interface
// values at the stage end (Eq. S2O3) and Gauss-theorem gradients (Eq. slope-1).
// Returns the CFL ratio dX/U_max of the new state (stage 2) or 0.
template <typename R>
__host__ __device__ inline double update_unit(const Dev &d, const Par &p, int j, int stage, int *flags) {
  const int N = d.cs, NE = d.ne;
  const int in = d.inst[j];
  const double dt = d.dt[in];
  // the unit's loads and arithmetic do not wait on dt: a cell of an instance
  // that has stopped (dt = 0) is computed too, and only its writes are dropped
  const bool act = dt > 0;
  const R *eF = (const R *)d.eF, *eFt = (const R *)d.eFt, *eWt = (const R *)d.eWt, *eWn = (const R *)d.eWn;
  const R *eO = (const R *)d.eO;
  const R *en = (const R *)d.en;
  const R dtr = ((const R *)d.dtR)[in];
  const R cend = stage == 1 ? (R)0.5 * dtr : dtr;
  // mass residuals in FP64 (exact conservation), the rest in R
  double LFm[2] = {0, 0}, LFtm[2] = {0, 0};
  R LF[NV] = {0}, LFt[NV] = {0}, mWt[NV] = {0};
  R GGt[NV][2] = {{0}}, GGn[NV][2] = {{0}};
  // the interlayer source's point values (R16): this cell's own levels at its
  // six Gauss points, their mean (mO) and Gauss-theorem gradient (GO), for
  // the lower (0: eta1 - R1) and upper (1: h2 - R2) layer
  R mO[2] = {0, 0}, GO[2][2] = {{0, 0}, {0, 0}};
  for (int f = 0; f < 3; f++) {
    int ce = d.cedge[f * N + j];
    int e = ce >= 0 ? ce : ~ce;
    const int side = ce >= 0 ? 0 : 2;
    const double sl = d.fsl[f * N + j];
    const R slR = ((const R *)d.fslR)[f * N + j];
    const R nx = en[e], ny = en[NE + e];
    const R snx = slR * nx, sny = slR * ny;
    for (int l = 0; l < 2; l++) {
      const R o = eO[(side + l) * NE + e];
      mO[l] += o * (R)(1.0 / 3.0);
      GO[l][0] += snx * o; GO[l][1] += sny * o;
    }
    for (int v = 0; v < NV; v++) {
      R Wt = eWt[v * NE + e], Wn = eWn[v * NE + e];
      if (v == 0 || v == 3) {
        LFm[v / 3] -= sl * d.eFm[(v / 3) * NE + e];
        LFtm[v / 3] -= sl * d.eFtm[(v / 3) * NE + e];
        mWt[v] += Wt * (R)(1.0 / 3.0);
        GGt[v][0] += snx * Wt; GGt[v][1] += sny * Wt;
      } else {
        LF[v] -= slR * eF[v * NE + e];
        LFt[v] -= slR * eFt[v * NE + e];
      }
      R We = Wn + cend * Wt;
      GGn[v][0] += snx * We; GGn[v][1] += sny * We;
    }
  }
  const R G = pv<R>(p.g, p.gf), chi = pv<R>(p.chi, p.chif);
  const R gb[2] = {((const R *)d.bgR)[j], ((const R *)d.bgR)[N + j]};
  const R *dq = (const R *)d.dq;
  const R R2 = ((const R *)d.refR)[2 * in];
  const R hrc = ((const R *)d.hrefc)[j];          // R1 - B_j
  const R m1 = hrc + mO[0], m2 = R2 + mO[1];       // means of h1, h2 over the 6 Gauss points
  const R LFh2 = (R)LFm[0], LFh1 = (R)LFm[1];
  R L[NV], Lt[NV];
  for (int k = 0; k < 2; k++) {
    // upper layer: -G h2 grad(B + h1) with h1 = eta1 - B at the points; the
    // time derivative by the product rule with the interface solution's W_t (R4)
    L[1 + k] = LF[1 + k] - G * (dq[j] - mO[1]) * gb[k] - G * m2 * GO[0][k];
    Lt[1 + k] = LFt[1 + k] - G * (LFh2 - mWt[0]) * gb[k] - G * mWt[0] * GO[0][k] - G * m2 * GGt[3][k];
    // lower layer: flux reference pressure + bottom source -> -G (eta1 - R1) grad B; interlayer -chi G h1 grad h2
    L[4 + k] = LF[4 + k] - G * dq[3 * N + j] * gb[k] - chi * G * m1 * GO[1][k];
    Lt[4 + k] = LFt[4 + k] - G * LFh1 * gb[k] - chi * G * (mWt[3] * GO[1][k] + m1 * GGt[0][k]);
  }
  // S2O4 (Eq. SWE-fully-discrete): stage 1 W* = W^n + dt/2 L^n + dt^2/8 L_t^n;
  // stage 2 W^{n+1} = W^n + dt L^n + dt^2/6 L_t^n + dt^2/3 L_t^*. The layer
  // depths (exact conservation) in FP64 throughout; the momenta's increments
  // in R (their residuals are R), each added to the FP64 state once
  const int mom[4] = {1, 2, 4, 5};
  double nw[NV];
  for (int m = 0; m < 2; m++) {
    const int v = 3 * m;
    const double a = d.avg[v * N + j];
    if (stage == 1) {
      if (act) {
        d.Wn[v * N + j] = a;
        d.Ln[v * N + j] = LFm[m];
        d.Ltn[v * N + j] = LFtm[m];
      }
      nw[v] = a + 0.5 * dt * LFm[m] + 0.125 * dt * dt * LFtm[m];
    } else {
      nw[v] = d.Wn[v * N + j] + dt * d.Ln[v * N + j] + dt * dt * (1.0 / 6.0) * d.Ltn[v * N + j] +
              dt * dt * (1.0 / 3.0) * LFtm[m];
    }
  }
  R *inc = (R *)d.incR;
  const R dt2 = dtr * dtr;
  for (int i = 0; i < 4; i++) {
    const int v = mom[i];
    const double a = d.avg[v * N + j];
    if (stage == 1) {
      if (act) {
        d.Wn[v * N + j] = a;
        inc[i * N + j] = dtr * L[v] + dt2 * (R)(1.0 / 6.0) * Lt[v];
      }
      nw[v] = a + (double)((R)0.5 * dtr * L[v] + (R)0.125 * dt2 * Lt[v]);
    } else {
      nw[v] = d.Wn[v * N + j] + (double)(inc[i * N + j] + dt2 * (R)(1.0 / 3.0) * Lt[v]);
    }
  }
  if (act) {
    R *dqw = (R *)d.dq, *dgw = (R *)d.dg;
    for (int v = 0; v < NV; v++) {
      d.avg[v * N + j] = nw[v];
      // the interface values of variable 3 are water levels: grad h1 = grad eta1 - grad B
      dgw[(2 * v) * N + j] = v == 3 ? GGn[v][0] - gb[0] : GGn[v][0];
      dgw[(2 * v + 1) * N + j] = v == 3 ? GGn[v][1] - gb[1] : GGn[v][1];
    }
    dqw[j] = (R)(nw[0] - d.ref[2 * in]);
    dqw[3 * N + j] = (R)((nw[3] + d.bmean[j]) - d.ref[2 * in + 1]);
    for (int i = 0; i < 4; i++) dqw[mom[i] * N + j] = (R)nw[mom[i]];
  }
  // health flags by integer tests on the bits (off the FP64 pipe)
  int fl = 0;
  for (int v = 0; v < NV; v++)
    if (!finite_bits(nw[v]) || !isfinite(GGn[v][0]) || !isfinite(GGn[v][1])) fl |= 2;
  if (!(dbits(nw[0]) > 0) || !(dbits(nw[3]) > 0)) fl |= 1;
  *flags = act ? fl : 0;
  if (stage != 2 || !act) return 0;
  return cfl_ratio<R>(nw, d.dX[j], G);
}

}  // namespace gks2l
