/*
 * gks2l -- GB300 (sm_103a) library for one explicit S2O4 stage of the compact
 * gas-kinetic scheme (GKS) for the two-layer shallow water equations (TLSWE)
 * on triangle meshes, after Zhao, Gan & Xu, arXiv 2306.04467.
 *
 * The problem statement the calls follow (Sec. 2.1, Eq. SWE-macro): a triangle
 * mesh, a bottom B, the per-layer depths and discharges W = (h2, h2U2, h2V2,
 * h1, h1U1, h1V1) with layer 1 the lower layer, the density ratio
 * chi = rho2/rho1, gravity G and the CFL number (Sec. 4) -> the state after n
 * stages of the two-stage fourth-order (S2O4) time stepping
 * (Eq. SWE-fully-discrete). The state is the cell averages AND their
 * cell-averaged gradients (Sec. 3.3, Eq. slope-1), which the scheme updates.
 *
 * Conventions
 *  - Every call returns 0 (GKS2L_OK) or a negative GKS2L_E* code; no call
 *    aborts. Device-side faults (negative depth, non-finite values) are
 *    recorded in a status word and reported by gks2l_stats / gks2l_advance.
 *  - Host arrays are read during the call and never retained. Device memory
 *    (the workspace) is allocated by the caller (e.g. a torch tensor), bound
 *    with gks2l_bind and never freed by the library.
 *  - State arrays are variable-major in the caller's cell order:
 *      avg[v * n_tri + j], grad[(v * 2 + d) * n_tri + j]   (d = 0: x, 1: y)
 *    The library renumbers cells internally (space-filling curve); all public
 *    state calls use the caller's order.
 *  - All work runs on the stream given to gks2l_bind; calls that return host
 *    data synchronise that stream.
 */
#ifndef GKS2L_H
#define GKS2L_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GKS2L_OK 0
#define GKS2L_EINVAL -1      /* bad argument (null pointer, size, parameter)        */
#define GKS2L_EMESH -2       /* mesh not usable (orientation, periodic match, LS)   */
#define GKS2L_ECUDA -3       /* a CUDA runtime call failed                          */
#define GKS2L_ESTATE -4      /* call out of order (not bound, no state)             */
#define GKS2L_ENEGDEPTH -5   /* a depth is or became <= 0 on the device             */
#define GKS2L_ENONFINITE -6  /* a non-finite value appeared on the device           */
#define GKS2L_ESPACE -7      /* workspace too small                                 */
#define GKS2L_ENOTIMPL -8
#define GKS2L_ETOOBIG -9     /* size beyond a fixed maximum (gks2l_cfl_mass_noalloc) */
#define GKS2L_ETIMEOUT -10   /* a bounded device wait (operator staging) gave up;  *
                              * the stage's results are not valid                  */

/* boundary kinds per triangle edge (edge k runs from tri[k] to tri[(k+1)%3]) */
#define GKS2L_BC_INTERIOR 0
#define GKS2L_BC_WALL 1      /* reflecting wall: mirror ghost (Sec. 4.6 walls)       */
#define GKS2L_BC_PERIODIC 2  /* matched with the opposite side by `period`           */

/* arithmetic forms */
#define GKS2L_FP64 0         /* every step in FP64                                   */
#define GKS2L_FP32 1         /* FP32 moments and reconstruction; FP64 for the base
                                values, the well-balanced flux/source cancellation
                                and the conservation sums                           */

/* troubled-cell indicator in the reconstruction */
#define GKS2L_INDICATOR_OFF 0   /* nonlinear WENO weights in every cell              */
#define GKS2L_INDICATOR_MLP 1   /* learned gate: cells it calls smooth take the
                                   linear (P3) reconstruction                        */

/* A triangle mesh (host memory, read during gks2l_create only).
 * xy: 2*n_vert vertex coordinates; tri: 3*n_tri vertex indices, counter-
 * clockwise; tri_bc: 3*n_tri boundary kinds (NULL: every boundary edge is a
 * wall); period: translation between matched periodic sides (0 if unused). */
typedef struct {
  int32_t n_vert;
  const double *xy;
  int32_t n_tri;
  const int32_t *tri;
  const int8_t *tri_bc;
  double period[2];
} gks2l_mesh;

/* Scheme parameters.
 * g, chi, cfl: gravity G, density ratio chi = rho2/rho1 (Eq. SWE-macro) and
 *   CFL number of dt = CFL dX / U_max (Sec. 4).
 * eps, eps_num: collision time tau = eps dt + eps_num |(hl^2-hr^2)/(hl^2+hr^2)| dt
 *   (Sec. 4; paper values 0.05 and 5).
 * weno_gamma_hi: linear weight of the P3 candidate (the three P1 candidates
 *   share the rest); weno_eps: smoothness regulariser, eps = weno_eps |Omega|
 *   (1 + Q0^2). The paper defers both to an external reference.
 * precision: GKS2L_FP64 or GKS2L_FP32.
 * indicator, indicator_threshold: troubled-cell gate (GKS2L_INDICATOR_*); a
 *   cell is called smooth when the gate's output is below the threshold.
 * staging_poll_limit: how long a reconstruction block waits for its operator
 *   tile to arrive in shared memory. 0 (the default) waits up to about one
 *   second; n > 0 polls at most n - 1 times, so 1 gives up at once. A block
 *   that gives up records GKS2L_ETIMEOUT, waits once more (up to one second)
 *   so that no copy outlives it, and writes nothing; a test sets 1 to raise
 *   the code without a fault.
 * positivity_floor: an option that is not in the paper (0, the default, is
 *   the method as the paper states it). With a fraction f in (0, 1): after
 *   each reconstruction, a layer whose depth at one of the cell's six edge
 *   Gauss points falls below f times its cell-average depth has its depth
 *   and discharge polynomials scaled toward their averages by one factor so
 *   that the least point depth is f times the average (averages unchanged),
 *   and in a layer whose point depths dip below half its average the edge
 *   solution's side velocities are bounded by the two cells' average
 *   velocities. It carries the paper's large-jump cases (Riemann problem II,
 *   the circular interface), on which the method as read reaches a vacuum at
 *   an interface state in its first steps. Runs with it take the plain
 *   reconstruction, interface and edge kernels at their default launch
 *   shapes (the gate, where on, still decides the linear cells). */
typedef struct {
  double g, chi, cfl;
  double eps, eps_num;
  double weno_gamma_hi, weno_eps;
  int32_t precision;
  int32_t indicator;
  float indicator_threshold;
  int32_t staging_poll_limit;
  double positivity_floor;
} gks2l_params;

/* Run statistics (FP64 sums taken on the device). */
typedef struct {
  double mass[2];        /* sum |Omega_j| h_j of the current state (summed when
                            the statistics are read), layer 1 (lower), layer 2 */
  double t;              /* simulated time of instance 0                        */
  double dt_last;        /* last step size of instance 0                        */
  int64_t stages_done;
  int32_t status;        /* 0 or a GKS2L_E* code raised on the device           */
  int32_t n_instances;
  double smooth_fraction;/* share of cell-stages the gate sent to the linear path */
} gks2l_stats_t;

typedef struct gks2l_ctx gks2l_ctx;

/* Fill p with the paper's defaults (G = 9.81, chi = 1, CFL = 0.5, eps = 0.05,
 * eps_num = 5) and this library's WENO reading (0.85, 1.0), FP64, no gate. */
int gks2l_default_params(gks2l_params *p);

/* Build a context for one mesh: geometry, compact stencils (Eq.
 * Recons-stencil) and least-squares operators (Eq. Recons-system), all in FP64
 * on the host. Copies the mesh. Returns GKS2L_EMESH for clockwise or
 * degenerate triangles or unmatched periodic edges. */
int gks2l_create(const gks2l_mesh *mesh, const gks2l_params *params, gks2l_ctx **out);

/* Build one context over several independent meshes (an ensemble): each
 * instance keeps its own time step and time; they advance together. */
int gks2l_create_ensemble(int32_t n, const gks2l_mesh *meshes, const gks2l_params *params,
                          gks2l_ctx **out);

/* Device bytes the caller must provide to gks2l_bind. */
int gks2l_workspace_bytes(const gks2l_ctx *ctx, size_t *bytes);

/* Bind caller-owned device memory (>= gks2l_workspace_bytes, 256-byte
 * aligned) and a CUDA stream (cudaStream_t, NULL = default stream); uploads
 * the mesh operators. The library never frees the workspace. */
int gks2l_bind(gks2l_ctx *ctx, void *d_workspace, size_t bytes, void *stream);

/* The bottom topography B of the source L^S1 (Sec. 3.2, Eq. SWE-semi-source:
 * h_j (0, -G B_x, -G B_y)) and of the water level h1 + B (Sec. 3.2's
 * well-balanced condition): the paper's "discretized bottom" (Sec. 4.2),
 * read here as B sampled at the vertices (host, n_vert doubles, concatenated
 * over instances for an ensemble), continuous and linear on each triangle.
 * May be called before or after gks2l_bind; a state must be set again after
 * it (GKS2L_ESTATE otherwise). */
int gks2l_set_bathymetry(gks2l_ctx *ctx, const double *b_vert);

/* Set the state: the cell averages W_j (Eq. SWE-cell-average) of the
 * variables of Eq. SWE-macro, (h2, h2U2, h2V2, h1, h1U1, h1V1), and their
 * cell-averaged gradients (the compact scheme's second set of unknowns,
 * Sec. 3.3, Eq. slope), from host arrays (avg: 6*n_tri, grad: 12*n_tri or
 * NULL for zero gradients) in the caller's order; resets time and step
 * counters. A depth <= 0 or a non-finite value is reported in the status
 * (GKS2L_ENEGDEPTH, GKS2L_ENONFINITE) that gks2l_stats and gks2l_advance
 * return; setting a good state clears it.
 * Each instance's reference levels (the area-weighted means of h2 and
 * h1 + B, rounded to 2^-32, about which the FP32 form computes deviations)
 * are reduced on the device in a fixed order. Returns after the host arrays
 * have been read (synchronises the stream). */
int gks2l_set_state(gks2l_ctx *ctx, const double *avg, const double *grad);
/* Same from device arrays (caller order), enqueued on the bound stream
 * without synchronising; the arrays must stay valid until the stream has
 * run it. */
int gks2l_set_state_device(gks2l_ctx *ctx, const double *d_avg, const double *d_grad);

/* Advance by up to n_stages stages (two stages make one S2O4 step). With
 * t_end > 0 each step is shortened to land on t_end and no step starts at or
 * after it; every 32 steps the call reads the instances' times back
 * (synchronising the stream) and returns once all have reached t_end, so a
 * large n_stages with an end time costs only the steps needed (plus at most
 * 31). Without t_end it only enqueues work on the bound stream. t_out (if not
 * NULL) forces a synchronisation and returns the time of instance 0. Returns
 * a device status code only when t_out is requested. */
int gks2l_advance(gks2l_ctx *ctx, int32_t n_stages, double t_end, double *t_out);

/* Copy the state (the averages and cell-averaged gradients of Eq. SWE-macro's
 * variables, as gks2l_set_state takes them) to host arrays (caller order);
 * synchronises the stream. A state read out and set again continues bit for
 * bit as if uninterrupted (plain forms; the gate restarts from the plain
 * method). */
int gks2l_get_state(gks2l_ctx *ctx, double *avg, double *grad);
/* Copy the state to device arrays (caller order) on the bound stream. */
int gks2l_get_state_device(gks2l_ctx *ctx, double *d_avg, double *d_grad);

/* Pipelined host I/O (not part of the paper): n_items independent states,
 * each set from host arrays as gks2l_set_state does, advanced n_stages
 * stages (no end time) and read back to host arrays as gks2l_get_state does,
 * in one call. Item i's host->device copy runs on an input copy stream and
 * its device->host copy on an output copy stream, so with pinned host memory
 * they overlap the computation of items i - 1 and i + 1 (pageable memory is
 * accepted; its copies then serialise with the computation).
 * in_avg[i], in_grad[i]: item i's state in the gks2l_set_state layout
 * (in_grad itself or in_grad[i] may be NULL: zero gradients); out_avg[i],
 * out_grad[i]: where its result goes, in the gks2l_get_state layout
 * (out_grad or out_grad[i] may be NULL). Host arrays must stay valid until
 * the call returns; an input and an output array must not overlap; one
 * output array may serve several items (the copies run in item order, the
 * last item's result remains). On return every copy has completed and the
 * context holds the last item's state, as after gks2l_set_state and
 * gks2l_advance. Returns GKS2L_EINVAL for n_items < 0, n_stages < 0 or a NULL
 * in_avg[i] / out_avg[i]; otherwise the combined status of all items
 * (GKS2L_ETIMEOUT, GKS2L_ENONFINITE, GKS2L_ENEGDEPTH as gks2l_advance).
 * The first call allocates four staging buffers of 18 doubles per cell and
 * two copy streams, kept until gks2l_destroy. */
int gks2l_run_items(gks2l_ctx *ctx, int32_t n_items, int32_t n_stages, const double *const *in_avg,
                    const double *const *in_grad, double *const *out_avg, double *const *out_grad);

/* Statistics: each layer's mass sum_j |Omega_j| h_j (the quantity the
 * finite-volume form Eq. SWE-semi-discrete conserves), the time and last
 * step (Sec. 4's CFL step), the stages done and the device status;
 * synchronises the stream. */
int gks2l_stats(gks2l_ctx *ctx, gks2l_stats_t *out);

/* ---- learned troubled-cell gate (not part of the paper) ------------------
 * A 24 -> 32 -> 32 -> 1 MLP (ReLU hidden layers, sigmoid output) predicts per
 * cell whether the nonlinear WENO weights of the reconstruction would depart
 * from the linear ones; cells it calls smooth take the linear P3
 * reconstruction and a blending weight w = 1. The network runs on a second
 * stream beside each stage's reconstruction or edge kernels, on the state
 * that stage reconstructed, and its decisions apply to the next
 * reconstruction; gks2l_set_state runs it once on the state it sets, for
 * the first stage (the first stage after gks2l_set_mlp is the plain
 * method). gks2l_set_mlp creates that stream. Parameters are a float vector
 * of GKS2L_MLP_NPARAM entries:
 *   W1[32][24], b1[32], W2[32][32], b2[32], w3[32], b3, mean[24], inv_std[24]
 * (the first GKS2L_MLP_NTRAIN are trained; features are (x - mean) * inv_std).
 * Weights run as BF16 on the tensor cores with FP32 accumulation. */
#define GKS2L_MLP_NPARAM 1937
#define GKS2L_MLP_NTRAIN 1889

/* Load the gate into a bound context (host params); it acts when the
 * context was created with indicator = GKS2L_INDICATOR_MLP. */
int gks2l_set_mlp(gks2l_ctx *ctx, const float *params, size_t n_floats);

/* Training data from the current state (after any number of stages), in the
 * caller's cell order: 24 features per cell d_features[24 * n_tri] and the
 * label d_labels[n_tri] = 1 where, in the plain nonlinear reconstruction of
 * the current state, max over the six variables and four WENO weights of
 * |omega_k / gamma_k - 1| exceeds tol. Features, columns 0-11 for eta1 and
 * 12-23 for h2: over the cell and its three face neighbours (face k is the
 * edge from vertex k to vertex k+1), the deviation of the average from the
 * four-cell mean and sqrt(|Omega|) times the gradient, divided by
 * sqrt(sum of their squares + weno_eps |Omega| (1 + q0^2)). d_logits: null,
 * or n_tri floats for the logits the fused gate computes for these cells
 * (needs a network loaded by gks2l_set_mlp). All pointers are device memory.
 * Synchronises the stream; the state is not changed (a gate loaded with
 * gks2l_set_mlp takes its decisions for the next stage from this state). */
int gks2l_harvest(gks2l_ctx *ctx, float tol, float *d_features, float *d_labels, float *d_logits);

/* Gradient of the weighted logistic loss
 *   L = sum_i pos_weight y_i softplus(-s_i) + (1 - y_i) softplus(s_i)
 * of n samples (device d_X[n][24], d_y[n] in {0, 1}) for parameters d_params
 * (device, GKS2L_MLP_NPARAM floats): writes d_grads[GKS2L_MLP_NTRAIN] (sums
 * over the samples) and d_loss[1]. BF16 tensor cores, FP32 sums in a fixed
 * order (the result is reproducible). Takes stream-ordered scratch of about
 * 7.6 KB per 64 samples (at most 18 MB). */
int gks2l_mlp_grad(const float *d_X, const float *d_y, int32_t n, const float *d_params, float pos_weight,
                   float *d_grads, float *d_loss, void *stream);

/* One Adam step (beta 0.9, 0.999, eps 1e-8) on the trained parameters with
 * gradients scaled by `scale`; step counts from 1. d_m, d_v: moment buffers of
 * GKS2L_MLP_NTRAIN floats, zero before the first step. */
int gks2l_mlp_adam(float *d_params, const float *d_grads, float *d_m, float *d_v, int32_t step, float lr,
                   float scale, void *stream);

/* Logits of n samples (device d_X[n][24]) with the tensor-core inference
 * path the reconstruction uses. */
int gks2l_mlp_forward(const float *d_X, int32_t n, const float *d_params, float *d_logits, void *stream);

/* ---- launch shapes (not part of the paper) --------------------------------
 * The interface, edge and update kernels each run in one of five launch
 * shapes (with the gate on, the edge shape applies to the fused interface and
 * edge kernel): 0: 64 threads per block, 1: 128 (default), 2: 256, 3: 128 threads
 * held to 64 registers (eight blocks per SM), 4: 128 threads held to 128
 * registers (four blocks per SM). shapes[3] picks the learned gate's variant:
 * its kernel (shapes[3] % 4): 0 (default), each warp takes 32 cells through
 * mma.sync BF16 tiles, the network in registers; 1, each 128-thread block
 * takes 128 cells through tcgen05 MMAs (M = 128, N = 32) with the
 * accumulators in tensor memory and the network in shared memory; 2 and 3,
 * the same kernel with two and four times as many blocks per SM. Its
 * placement (shapes[3] / 4 % 2): the gate reads the stage's state and runs on
 * a second stream beside the edge kernels (0) or beside the reconstruction
 * (1), joining before the cell update. The gated run's edge path
 * (shapes[3] / 8): 0, one fused interface-and-edge pass plus a deferred pass
 * for the edges whose plane gradients carry weight; 1, the plain interface
 * and edge kernels (faster when the gate calls few cells smooth). The gate
 * kernels may differ in the last bit of a logit; placement and edge path
 * change no result. */
#define GKS2L_LAUNCH_SHAPES 5
#define GKS2L_GATE_KERNELS 4
#define GKS2L_GATE_VARIANTS 16
int gks2l_set_launch_shapes(gks2l_ctx *ctx, const int32_t shapes[4]);

/* Autotuner: advances the state by GKS2L_LAUNCH_SHAPES * n_steps full steps,
 * exactly as gks2l_advance would, timing the interface, edge and update
 * kernels in each shape (CUDA events on the bound stream); keeps the fastest
 * for each. With the gate on it then times GKS2L_GATE_VARIANTS * (n_steps + 1)
 * more steps, whole steps per gate variant (the gate overlaps other kernels,
 * so its own time does not decide), and keeps the fastest. Writes the
 * choices to shapes[4]. Requires a state and phase at a step boundary;
 * returns the run's status like gks2l_advance with t_out. */
int gks2l_autotune(gks2l_ctx *ctx, int32_t n_steps, int32_t shapes[4]);

/* Kernel timing for roofline reports: advances n_steps full steps (exactly
 * like gks2l_advance, state included) but launches the stage kernels one by
 * one between CUDA events on the bound stream, then synchronises. ms[k] is
 * the mean duration of one launch of kernel k, in the order: reconstruction,
 * interface levels, edge solution, cell update (each averaged over both
 * stages), step start, troubled-cell gate (0 when it is off; run here in
 * sequence, in gks2l_advance on a second stream). With the gate on and the
 * fused edge path (gate variants 0-7), the
 * interface levels and the edge solution run as one fused kernel, reported
 * in the edge slot, followed by a pass over the edges whose solution needs
 * the plane gradients, reported in the interface slot.
 * Requires a state and phase at a step boundary. */
int gks2l_profile_kernels(gks2l_ctx *ctx, int32_t n_steps, double ms[6]);

/* Measurement helper with no counterpart in the paper: FP32 and FP64 FMA
 * throughput of the bound device (TFLOP/s, FMA = 2 flops) from FMA-chain
 * kernels on the bound stream, the denominators of the ALU rooflines.
 * Uses the context's staging area (needs n_tri >= 8 * SMs * 256 / 18). */
int gks2l_alu_peaks(gks2l_ctx *ctx, double tflops[2]);

/* CFL step and layer masses of a device state, allocating nothing.
 * The paper has no counterpart: this is a service for callers that cannot
 * call cudaMalloc -- code running inside another framework's memory pool, a
 * process whose device memory is fully reserved up front, or a loop that must
 * not allocate -- and so cannot provide the workspace gks2l_bind needs. It
 * computes what the library's own CFL kernel computes for a bound context
 * (Sec. 4: dt = CFL * min_j dX_j / U_max,j, U_max = max over layers of
 * |U| + sqrt(G h); plus sum_j |Omega_j| h_j per layer), with its scratch in a
 * fixed device array of 4 x 1024 doubles (32 KB) that every GPU loading the
 * library holds until the process exits.
 *   n_tri   number of cells, 1 .. GKS2L_NOALLOC_MAX_TRI (larger: GKS2L_ETOOBIG)
 *   d_avg   device, 6*n_tri doubles, variable-major state (any cell order)
 *   d_area  device, n_tri cell areas, d_dX device, n_tri CFL lengths
 *           (4 |Omega| / perimeter), both in the same cell order as d_avg
 *   d_out   device, 4 doubles written: dt, mass of layer 1 (lower), mass of
 *           layer 2, and the number of unusable cells (a depth <= 0 or a
 *           non-finite speed or CFL ratio); those cells take no part in dt
 *           (dt = inf if every cell is unusable), so a caller checks d_out[3]
 *           before trusting dt
 *   stream  cudaStream_t (NULL = default stream); the call only enqueues work.
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture. The address is kept for the life of the
 * process: after a cudaDeviceReset of that device it is stale, so calls after
 * a reset are not supported (they would launch kernels on an unmapped
 * address). All calls share the one array, so calls whose
 * work overlaps on the GPU (other streams, other threads) race; serialise
 * them. Nothing in the array needs clearing: each call overwrites the slots it
 * reads. Calls no cudaMalloc, cudaFree or allocating library routine. */
#define GKS2L_NOALLOC_MAX_TRI (1 << 28)
int gks2l_cfl_mass_noalloc(int32_t n_tri, const double *d_avg, const double *d_area, const double *d_dX,
                           double g, double cfl, double *d_out, void *stream);

/* Human-readable name of a status code. */
const char *gks2l_error_string(int code);

void gks2l_destroy(gks2l_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif
