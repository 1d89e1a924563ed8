/*
 * ORACLE -- test infrastructure only.
 *
 * A plain, slow, serial FP64 CPU restatement of the compact gas-kinetic scheme
 * (GKS) for the two-layer shallow water equations on triangles of
 * Zhao, Gan & Xu, "High-order compact gas-kinetic scheme for two-layer shallow
 * water equations on unstructured mesh" (arXiv 2306.04467). It exists to check
 * the CUDA path: only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline may load it. It shares no code with the CUDA library.
 *
 * Every routine follows the paper's steps in its notation; where the paper is
 * silent the reading is named (R1..R20) and listed with its reason in the
 * repository's design notes. Build: gcc -O2 -ffp-contract=off -fPIC -shared.
 *
 * Variable order per cell (Sec. 2.1, Eq. SWE-macro): h2, h2U2, h2V2, h1, h1U1,
 * h1V1; layer 1 is the lower layer, layer 2 the upper one.
 *
 * Parity notes: every routine here is pinned by a CPU test (moments and time
 * integrals against quadrature, the point solution against brute-force
 * velocity/time quadrature, cubic reproduction, Gauss-theorem exactness,
 * uniform flux, lake at rest, conservation, convergence order). The blend
 * of Sec. 2.3 is pinned in its closed-form cases (xi = 1/2 at rest, xi = 0
 * or 1 in strong flow, against the two sides' point values) and the planes
 * through the blended levels (exact for linear levels). The WENO constants
 * (R5) and the form of the edge weight w (R6) are not fixed by the paper:
 * for them parity is unpinned against the paper (parity unpinned), fixed by
 * the readings and by the weights' pinned behaviour (exactly linear on
 * smooth data, collapsing at a jump).
 *
 * One addition is not in the paper: an off-by-default positivity option
 * (orc_set_positivity; positivity_scale and the velocity bound in the edge
 * loop) for the large-jump cases the method as read cannot carry. It is
 * pinned by a smooth flow it leaves unchanged bit for bit and by Riemann
 * problem II's conservation and bounds.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define NVAR 6
#define MAXAVG 9          /* averages rows of the P3 system (Eq. Recons-system) */
#define MAXROWS 17        /* 9 average rows + 8 gradient rows                 */
#define NB 10             /* P3 basis size (Eq. Recons-poly)                   */

enum { BC_INTERIOR = 0, BC_WALL = 1, BC_PERIODIC = 2 };

/* ------------------------------------------------------------------------- */
/* affine isometries x' = m x + t used for periodic images and wall mirrors   */
/* ------------------------------------------------------------------------- */
typedef struct { double m[2][2]; double t[2]; } aff_t;

static aff_t aff_id(void) { aff_t a = {{{1, 0}, {0, 1}}, {0, 0}}; return a; }
static aff_t aff_shift(double sx, double sy) { aff_t a = aff_id(); a.t[0] = sx; a.t[1] = sy; return a; }
/* mirror across the line through p with unit normal n */
static aff_t aff_mirror(const double p[2], const double n[2]) {
  aff_t a;
  a.m[0][0] = 1 - 2 * n[0] * n[0]; a.m[0][1] = -2 * n[0] * n[1];
  a.m[1][0] = -2 * n[1] * n[0];    a.m[1][1] = 1 - 2 * n[1] * n[1];
  double pn = p[0] * n[0] + p[1] * n[1];
  a.t[0] = 2 * pn * n[0]; a.t[1] = 2 * pn * n[1];
  return a;
}
/* (a o b)(x) = a(b(x)) */
static aff_t aff_compose(const aff_t *a, const aff_t *b) {
  aff_t c;
  for (int i = 0; i < 2; i++) {
    for (int j = 0; j < 2; j++) c.m[i][j] = a->m[i][0] * b->m[0][j] + a->m[i][1] * b->m[1][j];
    c.t[i] = a->m[i][0] * b->t[0] + a->m[i][1] * b->t[1] + a->t[i];
  }
  return c;
}
static void aff_apply(const aff_t *a, const double x[2], double y[2]) {
  double y0 = a->m[0][0] * x[0] + a->m[0][1] * x[1] + a->t[0];
  double y1 = a->m[1][0] * x[0] + a->m[1][1] * x[1] + a->t[1];
  y[0] = y0; y[1] = y1;
}
/* inverse of an isometry: m^T (y - t) */
static void aff_apply_inv(const aff_t *a, const double y[2], double x[2]) {
  double d0 = y[0] - a->t[0], d1 = y[1] - a->t[1];
  x[0] = a->m[0][0] * d0 + a->m[1][0] * d1;
  x[1] = a->m[0][1] * d0 + a->m[1][1] * d1;
}
static void rot_vec(const aff_t *a, const double v[2], double out[2]) {
  double o0 = a->m[0][0] * v[0] + a->m[0][1] * v[1];
  double o1 = a->m[1][0] * v[0] + a->m[1][1] * v[1];
  out[0] = o0; out[1] = o1;
}

typedef struct { int cell; aff_t T; } image_t;   /* a cell seen through T */

/* ------------------------------------------------------------------------- */
/* quadrature on a triangle: collapsed 3x3 Gauss-Legendre rule, exact for     */
/* total degree <= 4 (the cubic basis averages and the squared derivatives   */
/* of the smoothness indicator need degree 3 and 4).                          */
/* ------------------------------------------------------------------------- */
#define NQT 9
static double QT_A[NQT], QT_B[NQT], QT_W[NQT];   /* barycentric (a,b), weights summing to 1 */
static void quad_init(void) {
  static int done = 0;
  if (done) return;
  const double g[3] = {0.5 - 0.5 * sqrt(0.6), 0.5, 0.5 + 0.5 * sqrt(0.6)};
  const double w[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
  double sum = 0;
  int k = 0;
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++, k++) {
      QT_A[k] = g[i];
      QT_B[k] = g[j] * (1 - g[i]);
      QT_W[k] = w[i] * w[j] * (1 - g[i]);
      sum += QT_W[k];
    }
  for (k = 0; k < NQT; k++) QT_W[k] /= sum;
  done = 1;
}

/* ------------------------------------------------------------------------- */
/* P3 basis (Eq. Recons-poly / Recons-eqs): Taylor monomials in the scaled    */
/* coordinates xi = (x - x_c)/h, h = sqrt(|Omega|) (reading R9), made zero-   */
/* mean over the own cell.                                                   */
/* ------------------------------------------------------------------------- */
static void monomials(double x, double y, double m[NB]) {
  m[0] = 1; m[1] = x; m[2] = y;
  m[3] = 0.5 * x * x; m[4] = x * y; m[5] = 0.5 * y * y;
  m[6] = x * x * x / 6; m[7] = 0.5 * x * x * y; m[8] = 0.5 * x * y * y; m[9] = y * y * y / 6;
}
static void monomials_dx(double x, double y, double m[NB]) {
  m[0] = 0; m[1] = 1; m[2] = 0;
  m[3] = x; m[4] = y; m[5] = 0;
  m[6] = 0.5 * x * x; m[7] = x * y; m[8] = 0.5 * y * y; m[9] = 0;
}
static void monomials_dy(double x, double y, double m[NB]) {
  m[0] = 0; m[1] = 0; m[2] = 1;
  m[3] = 0; m[4] = x; m[5] = y;
  m[6] = 0; m[7] = 0.5 * x * x; m[8] = x * y; m[9] = 0.5 * y * y;
}

/* ------------------------------------------------------------------------- */
/* the oracle context                                                        */
/* ------------------------------------------------------------------------- */
typedef struct {
  int L;           /* left cell: the edge runs counter-clockwise around L    */
  int kL;          /* local edge index in L                                  */
  int bc;          /* BC_INTERIOR, BC_WALL or BC_PERIODIC                    */
  image_t R;       /* right cell as seen from L's frame (mirror of L at walls) */
  double n[2];     /* unit normal from L to R                                */
  double len;
  double xq[2][2]; /* Gauss points, L's frame                                */
  double bq[2];    /* bathymetry at the Gauss points                         */
  double mid[2];   /* edge centre, L's frame                                 */
} edge_t;

typedef struct {
  int nv, nt, ne;
  double *xy; int *tri; signed char *tri_bc;
  double period[2];
  double g, chi, cfl, eps, eps_num, gam_hi, weno_eps;
  double pos_floor;                      /* positivity option (not in the paper): 0 = off */
  unsigned char *pos_scaled;             /* 2 per cell: layer (0 lower, 1 upper) scaled this stage */
  /* geometry per cell */
  double *area, *cx, *cy, *hs, *dX, *bmean;  /* bmean: cell average of the P1 bottom */
  double *bgrad;                         /* 2 per cell */
  double *bvert;
  double *mean_m;                        /* NB per cell: mean of each monomial over the cell (xi coords) */
  image_t *face;                         /* 3 per cell: images across the cell's edges */
  int *face_edge, *face_side;            /* edge id and side (+1: cell is L, -1: cell is R) */
  /* LS operators per cell */
  int *navg;                             /* number of average rows */
  image_t *avg_img;                      /* MAXAVG per cell */
  double *M;                             /* 9 x MAXROWS per cell (pseudo-inverse) */
  double *N1;                            /* 3 sub-stencils x 2 x 5 per cell */
  edge_t *edge;
  /* state */
  double *avg, *grad;                    /* avg[j*6+v], grad[(j*6+v)*2+d] */
  double t, dt;
  int phase;                             /* 0: next stage is stage 1; 1: stage 2 */
  long long stages_done;
  /* stage work arrays */
  double *coef;                          /* NB per (cell,var): reconstructed polynomial */
  double *omegaH;                        /* per (cell,var): nonlinear weight of the P3 candidate */
  double *wdev;                          /* per (cell,var): max_k |omega_k / gamma_k - 1|        */
  unsigned char *linear;                 /* per cell: 1 = take the linear weights (gate), or NULL */
  double *hc;                            /* per edge: edge-centre blended heights, layer 1 (depth), layer 2 */
  double *plane;                         /* per cell: grad of the P1 plane of h1_hat (2) and h2_hat (2) */
  double *eF, *eFt, *eW, *eWt;           /* per edge per Gauss point: 6 each, global frame */
  double *eWn;                           /* stage-1 interface values W^n(x) */
  double *Wn, *Ln, *Ltn;                 /* stage snapshot per cell */
  int status;
} orc_t;

#define IDX2(j, k) ((j) * 3 + (k))


/* ---- mean over a triangle (given by 3 vertices) of the basis of cell j -- */
static void cell_to_xi(const orc_t *o, int j, const double x[2], double xi[2]) {
  xi[0] = (x[0] - o->cx[j]) / o->hs[j];
  xi[1] = (x[1] - o->cy[j]) / o->hs[j];
}

/* average over triangle P of monomials (and their xi-derivatives) of cell j */
static void tri_avg_monomials(const orc_t *o, int j, const double P[3][2],
                              double am[NB], double adx[NB], double ady[NB]) {
  quad_init();
  for (int k = 0; k < NB; k++) am[k] = adx[k] = ady[k] = 0;
  for (int q = 0; q < NQT; q++) {
    double x[2], xi[2], m[NB], mx[NB], my[NB];
    x[0] = P[0][0] + QT_A[q] * (P[1][0] - P[0][0]) + QT_B[q] * (P[2][0] - P[0][0]);
    x[1] = P[0][1] + QT_A[q] * (P[1][1] - P[0][1]) + QT_B[q] * (P[2][1] - P[0][1]);
    cell_to_xi(o, j, x, xi);
    monomials(xi[0], xi[1], m);
    monomials_dx(xi[0], xi[1], mx);
    monomials_dy(xi[0], xi[1], my);
    for (int k = 0; k < NB; k++) {
      am[k] += QT_W[q] * m[k];
      adx[k] += QT_W[q] * mx[k];
      ady[k] += QT_W[q] * my[k];
    }
  }
}

static void cell_vertices(const orc_t *o, int c, double P[3][2]) {
  for (int k = 0; k < 3; k++) {
    P[k][0] = o->xy[2 * o->tri[3 * c + k]];
    P[k][1] = o->xy[2 * o->tri[3 * c + k] + 1];
  }
}
static void image_vertices(const orc_t *o, const image_t *im, double P[3][2]) {
  double Q[3][2];
  cell_vertices(o, im->cell, Q);
  for (int k = 0; k < 3; k++) aff_apply(&im->T, Q[k], P[k]);
}
static void image_centroid(const orc_t *o, const image_t *im, double c[2]) {
  double x[2] = {o->cx[im->cell], o->cy[im->cell]};
  aff_apply(&im->T, x, c);
}

/* ------------------------------------------------------------------------- */
/* least squares: pseudo-inverse by Householder QR of an m x n matrix (m>=n) */
/* The paper writes a = (A^T A)^-1 A^T Q; QR gives the same operator without */
/* squaring the condition number.                                             */
/* ------------------------------------------------------------------------- */
static int pinv_qr(int m, int n, const double *A /* m x n row-major */, double *P /* n x m */) {
  double R[MAXROWS][NB], Qt[MAXROWS][MAXROWS];
  for (int i = 0; i < m; i++) {
    for (int j = 0; j < n; j++) R[i][j] = A[i * n + j];
    for (int j = 0; j < m; j++) Qt[i][j] = (i == j);
  }
  for (int k = 0; k < n; k++) {
    double nrm = 0;
    for (int i = k; i < m; i++) nrm += R[i][k] * R[i][k];
    nrm = sqrt(nrm);
    if (nrm == 0) return -1;
    double alpha = R[k][k] > 0 ? -nrm : nrm;
    double v[MAXROWS];
    for (int i = 0; i < m; i++) v[i] = 0;
    v[k] = R[k][k] - alpha;
    for (int i = k + 1; i < m; i++) v[i] = R[i][k];
    double vv = 0;
    for (int i = k; i < m; i++) vv += v[i] * v[i];
    if (vv == 0) continue;
    for (int j = 0; j < n; j++) {
      double s = 0;
      for (int i = k; i < m; i++) s += v[i] * R[i][j];
      s = 2 * s / vv;
      for (int i = k; i < m; i++) R[i][j] -= s * v[i];
    }
    for (int j = 0; j < m; j++) {
      double s = 0;
      for (int i = k; i < m; i++) s += v[i] * Qt[i][j];
      s = 2 * s / vv;
      for (int i = k; i < m; i++) Qt[i][j] -= s * v[i];
    }
  }
  /* A = Q R, so pinv = R^-1 (Q^T)[0:n, :] */
  for (int c = 0; c < m; c++) {
    for (int i = n - 1; i >= 0; i--) {
      double s = Qt[i][c];
      for (int j = i + 1; j < n; j++) s -= R[i][j] * P[j * m + c];
      if (R[i][i] == 0) return -1;
      P[i * m + c] = s / R[i][i];
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* mesh set-up: geometry, edges (unique, periodic pairs matched), images     */
/* ------------------------------------------------------------------------- */
typedef struct { int a, b, cell, k; } hedge_t;
static int hedge_cmp(const void *x, const void *y) {
  const hedge_t *p = x, *q = y;
  if (p->a != q->a) return p->a < q->a ? -1 : 1;
  if (p->b != q->b) return p->b < q->b ? -1 : 1;
  return 0;
}

static void edge_geometry(const orc_t *o, int c, int k, double pa[2], double pb[2]) {
  int va = o->tri[3 * c + k], vb = o->tri[3 * c + (k + 1) % 3];
  pa[0] = o->xy[2 * va]; pa[1] = o->xy[2 * va + 1];
  pb[0] = o->xy[2 * vb]; pb[1] = o->xy[2 * vb + 1];
}

static int same_point(const double *p, const double *q, double tol) {
  return fabs(p[0] - q[0]) <= tol && fabs(p[1] - q[1]) <= tol;
}

/* images equal if they show the same cell at the same place */
static int same_image(const orc_t *o, const image_t *a, const image_t *b, double tol) {
  if (a->cell != b->cell) return 0;
  double ca[2], cb[2];
  image_centroid(o, a, ca);
  image_centroid(o, b, cb);
  return same_point(ca, cb, tol);
}

static int build_mesh(orc_t *o) {
  int nt = o->nt;
  /* per-cell geometry */
  for (int c = 0; c < nt; c++) {
    double P[3][2];
    cell_vertices(o, c, P);
    double a = 0.5 * ((P[1][0] - P[0][0]) * (P[2][1] - P[0][1]) - (P[1][1] - P[0][1]) * (P[2][0] - P[0][0]));
    if (!(a > 0)) return -2;
    o->area[c] = a;
    o->cx[c] = (P[0][0] + P[1][0] + P[2][0]) / 3;
    o->cy[c] = (P[0][1] + P[1][1] + P[2][1]) / 3;
    o->hs[c] = sqrt(a);
    double per = 0;
    for (int k = 0; k < 3; k++) per += hypot(P[(k + 1) % 3][0] - P[k][0], P[(k + 1) % 3][1] - P[k][1]);
    o->dX[c] = 4 * a / per;               /* reading R10: inscribed-circle diameter */
  }
  /* edges: interior pairs by sorting vertex pairs */
  hedge_t *he = malloc(sizeof(hedge_t) * 3 * nt);
  for (int c = 0; c < nt; c++)
    for (int k = 0; k < 3; k++) {
      int va = o->tri[3 * c + k], vb = o->tri[3 * c + (k + 1) % 3];
      he[3 * c + k].a = va < vb ? va : vb;
      he[3 * c + k].b = va < vb ? vb : va;
      he[3 * c + k].cell = c;
      he[3 * c + k].k = k;
    }
  qsort(he, 3 * nt, sizeof(hedge_t), hedge_cmp);
  o->edge = calloc((size_t)3 * (size_t)nt, sizeof(edge_t));
  int ne = 0;
  int *bnd = malloc(sizeof(int) * 3 * nt), nb = 0;   /* boundary half-edges */
  for (int i = 0; i < 3 * nt;) {
    if (i + 1 < 3 * nt && he[i].a == he[i + 1].a && he[i].b == he[i + 1].b) {
      edge_t *e = &o->edge[ne];
      /* L: the cell with the lower index */
      int c0 = he[i].cell, k0 = he[i].k, c1 = he[i + 1].cell, k1 = he[i + 1].k;
      if (c1 < c0) { int t = c0; c0 = c1; c1 = t; t = k0; k0 = k1; k1 = t; }
      e->L = c0; e->kL = k0; e->bc = BC_INTERIOR;
      e->R.cell = c1; e->R.T = aff_id();
      o->face[IDX2(c0, k0)] = (image_t){c1, aff_id()};
      o->face[IDX2(c1, k1)] = (image_t){c0, aff_id()};
      o->face_edge[IDX2(c0, k0)] = ne; o->face_side[IDX2(c0, k0)] = +1;
      o->face_edge[IDX2(c1, k1)] = ne; o->face_side[IDX2(c1, k1)] = -1;
      ne++;
      i += 2;
    } else {
      bnd[nb++] = 3 * he[i].cell + he[i].k;
      i += 1;
    }
  }
  free(he);
  /* boundary edges: walls mirror the cell; periodic ones are matched by translation */
  char *used = calloc(nb, 1);
  for (int i = 0; i < nb; i++) {
    if (used[i]) continue;
    int c = bnd[i] / 3, k = bnd[i] % 3;
    int kind = o->tri_bc ? o->tri_bc[3 * c + k] : BC_WALL;
    double pa[2], pb[2];
    edge_geometry(o, c, k, pa, pb);
    double mid[2] = {0.5 * (pa[0] + pb[0]), 0.5 * (pa[1] + pb[1])};
    double tol = 1e-9 * o->hs[c];
    if (kind == BC_PERIODIC) {
      int found = -1;
      double shift[2] = {0, 0};
      for (int j = i + 1; j < nb && found < 0; j++) {
        if (used[j]) continue;
        int c2 = bnd[j] / 3, k2 = bnd[j] % 3;
        double qa[2], qb[2];
        edge_geometry(o, c2, k2, qa, qb);
        double m2[2] = {0.5 * (qa[0] + qb[0]), 0.5 * (qa[1] + qb[1])};
        const double cand[4][2] = {{o->period[0], 0}, {-o->period[0], 0}, {0, o->period[1]}, {0, -o->period[1]}};
        for (int s = 0; s < 4; s++) {
          if (cand[s][0] == 0 && cand[s][1] == 0) continue;
          double mm[2] = {m2[0] + cand[s][0], m2[1] + cand[s][1]};
          if (same_point(mm, mid, tol)) { found = j; shift[0] = cand[s][0]; shift[1] = cand[s][1]; break; }
        }
      }
      if (found < 0) { free(bnd); free(used); return -3; }
      used[i] = used[found] = 1;
      int c2 = bnd[found] / 3, k2 = bnd[found] % 3;
      /* L is the lower cell index; the other is seen shifted */
      int cL = c, kLl = k, cR = c2, kRr = k2;
      double sR[2] = {shift[0], shift[1]};          /* maps cR's frame into cL's frame */
      if (c2 < c) { cL = c2; kLl = k2; cR = c; kRr = k; sR[0] = -shift[0]; sR[1] = -shift[1]; }
      edge_t *e = &o->edge[ne];
      e->L = cL; e->kL = kLl; e->bc = BC_PERIODIC;
      e->R.cell = cR; e->R.T = aff_shift(sR[0], sR[1]);
      o->face[IDX2(cL, kLl)] = (image_t){cR, aff_shift(sR[0], sR[1])};
      o->face[IDX2(cR, kRr)] = (image_t){cL, aff_shift(-sR[0], -sR[1])};
      o->face_edge[IDX2(cL, kLl)] = ne; o->face_side[IDX2(cL, kLl)] = +1;
      o->face_edge[IDX2(cR, kRr)] = ne; o->face_side[IDX2(cR, kRr)] = -1;
      ne++;
    } else {
      used[i] = 1;
      double d[2] = {pb[0] - pa[0], pb[1] - pa[1]};
      double l = hypot(d[0], d[1]);
      double n[2] = {d[1] / l, -d[0] / l};
      edge_t *e = &o->edge[ne];
      e->L = c; e->kL = k; e->bc = BC_WALL;
      e->R.cell = c; e->R.T = aff_mirror(pa, n);
      o->face[IDX2(c, k)] = e->R;
      o->face_edge[IDX2(c, k)] = ne; o->face_side[IDX2(c, k)] = +1;
      ne++;
    }
  }
  free(bnd); free(used);
  o->ne = ne;
  /* per-edge geometry, in L's frame */
  const double gs[2] = {0.5 - 0.5 / sqrt(3.0), 0.5 + 0.5 / sqrt(3.0)};
  for (int i = 0; i < ne; i++) {
    edge_t *e = &o->edge[i];
    double pa[2], pb[2];
    edge_geometry(o, e->L, e->kL, pa, pb);
    double d[2] = {pb[0] - pa[0], pb[1] - pa[1]};
    e->len = hypot(d[0], d[1]);
    e->n[0] = d[1] / e->len; e->n[1] = -d[0] / e->len;
    int va = o->tri[3 * e->L + e->kL], vb = o->tri[3 * e->L + (e->kL + 1) % 3];
    for (int q = 0; q < 2; q++) {
      e->xq[q][0] = pa[0] + gs[q] * d[0];
      e->xq[q][1] = pa[1] + gs[q] * d[1];
      e->bq[q] = o->bvert[va] + gs[q] * (o->bvert[vb] - o->bvert[va]);   /* R2: B linear along the edge */
    }
    e->mid[0] = 0.5 * (pa[0] + pb[0]); e->mid[1] = 0.5 * (pa[1] + pb[1]);
  }
  return 0;
}

/* bathymetry (reading R2): continuous piecewise-linear on the vertices */
static void build_bathymetry(orc_t *o) {
  for (int c = 0; c < o->nt; c++) {
    double P[3][2], b[3];
    cell_vertices(o, c, P);
    for (int k = 0; k < 3; k++) b[k] = o->bvert[o->tri[3 * c + k]];
    o->bmean[c] = (b[0] + b[1] + b[2]) / 3;
    double d1[2] = {P[1][0] - P[0][0], P[1][1] - P[0][1]};
    double d2[2] = {P[2][0] - P[0][0], P[2][1] - P[0][1]};
    double det = d1[0] * d2[1] - d1[1] * d2[0];
    double f1 = b[1] - b[0], f2 = b[2] - b[0];
    o->bgrad[2 * c] = (f1 * d2[1] - f2 * d1[1]) / det;
    o->bgrad[2 * c + 1] = (f2 * d1[0] - f1 * d2[0]) / det;
  }
  for (int i = 0; i < o->ne; i++) {
    edge_t *e = &o->edge[i];
    const double gs[2] = {0.5 - 0.5 / sqrt(3.0), 0.5 + 0.5 / sqrt(3.0)};
    int va = o->tri[3 * e->L + e->kL], vb = o->tri[3 * e->L + (e->kL + 1) % 3];
    for (int q = 0; q < 2; q++) e->bq[q] = o->bvert[va] + gs[q] * (o->bvert[vb] - o->bvert[va]);
  }
}

/* ------------------------------------------------------------------------- */
/* compact stencil and LS operators (Eqs. Recons-stencil, Recons-system)     */
/* ------------------------------------------------------------------------- */
static int build_operators(orc_t *o) {
  for (int j = 0; j < o->nt; j++) {
    double P[3][2], am[NB], adx[NB], ady[NB];
    cell_vertices(o, j, P);
    tri_avg_monomials(o, j, P, am, adx, ady);
    for (int k = 0; k < NB; k++) o->mean_m[j * NB + k] = am[k];
    double tol = 1e-8 * o->hs[j];
    /* stencil S0: face neighbours i, j, k, then their other neighbours (R8) */
    image_t list[MAXAVG];
    int n = 0;
    image_t self = {j, aff_id()};
    for (int f = 0; f < 3; f++) list[n++] = o->face[IDX2(j, f)];
    for (int f = 0; f < 3; f++) {
      image_t fi = o->face[IDX2(j, f)];
      for (int g = 0; g < 3; g++) {
        image_t nn = o->face[IDX2(fi.cell, g)];
        image_t cand = {nn.cell, aff_compose(&fi.T, &nn.T)};
        if (same_image(o, &cand, &self, tol)) continue;
        int dup = 0;
        for (int s = 0; s < n; s++) if (same_image(o, &cand, &list[s], tol)) { dup = 1; break; }
        if (dup) continue;
        if (n >= MAXAVG) return -4;
        list[n++] = cand;
      }
    }
    o->navg[j] = n;
    for (int s = 0; s < n; s++) o->avg_img[j * MAXAVG + s] = list[s];
    /* matrix rows: averages of the zero-mean basis over the image cells,   */
    /* then h-scaled average derivatives over the own cell and faces         */
    int m = n + 8;
    double A[MAXROWS * 9];
    for (int s = 0; s < n; s++) {
      double Q[3][2], im[NB], ix[NB], iy[NB];
      image_vertices(o, &list[s], Q);
      tri_avg_monomials(o, j, Q, im, ix, iy);
      for (int k = 1; k < NB; k++) A[s * 9 + (k - 1)] = im[k] - am[k];
    }
    for (int f = 0; f < 4; f++) {
      double Q[3][2], im[NB], ix[NB], iy[NB];
      if (f == 0) cell_vertices(o, j, Q);
      else image_vertices(o, &o->face[IDX2(j, f - 1)], Q);
      tri_avg_monomials(o, j, Q, im, ix, iy);
      for (int k = 1; k < NB; k++) {
        A[(n + 2 * f) * 9 + (k - 1)] = ix[k];
        A[(n + 2 * f + 1) * 9 + (k - 1)] = iy[k];
      }
    }
    double Pm[9 * MAXROWS];
    if (pinv_qr(m, 9, A, Pm)) return -5;
    /* store as 9 x MAXROWS with the gradient columns at the fixed places 9..16 */
    double *Mj = &o->M[j * 9 * MAXROWS];
    for (int r = 0; r < 9; r++) {
      for (int c = 0; c < MAXROWS; c++) Mj[r * MAXROWS + c] = 0;
      for (int c = 0; c < n; c++) Mj[r * MAXROWS + c] = Pm[r * m + c];
      for (int c = 0; c < 8; c++) Mj[r * MAXROWS + 9 + c] = Pm[r * m + n + c];
    }
    /* P1 sub-stencils (reading R5): cell j and face neighbour f */
    for (int f = 0; f < 3; f++) {
      double Q[3][2], im[NB], ix[NB], iy[NB];
      image_vertices(o, &o->face[IDX2(j, f)], Q);
      tri_avg_monomials(o, j, Q, im, ix, iy);
      double B5[5 * 2] = {im[1] - am[1], im[2] - am[2], 1, 0, 0, 1, 1, 0, 0, 1};
      double P5[2 * 5];
      if (pinv_qr(5, 2, B5, P5)) return -6;
      for (int i = 0; i < 10; i++) o->N1[(j * 3 + f) * 10 + i] = P5[i];
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* cell data as seen through an image transform                              */
/* reconstructed variables: h2, m2x, m2y, eta1 = h1 + B (water-level          */
/* reconstruction, Sec. 3.2), m1x, m1y                                       */
/* ------------------------------------------------------------------------- */
static void image_avg(const orc_t *o, const image_t *im, double q[NVAR]) {
  const double *a = &o->avg[im->cell * NVAR];
  q[0] = a[0]; q[3] = a[3] + o->bmean[im->cell];
  rot_vec(&im->T, &a[1], &q[1]);
  rot_vec(&im->T, &a[4], &q[4]);
}
/* gradients (d/dx, d/dy) of the reconstructed variables, image frame */
static void image_grad(const orc_t *o, const image_t *im, double gq[NVAR][2]) {
  const double *g = &o->grad[im->cell * NVAR * 2];
  double gr[NVAR][2];
  for (int v = 0; v < NVAR; v++) { gr[v][0] = g[2 * v]; gr[v][1] = g[2 * v + 1]; }
  gr[3][0] += o->bgrad[2 * im->cell];
  gr[3][1] += o->bgrad[2 * im->cell + 1];
  const aff_t *T = &im->T;
  for (int v = 0; v < NVAR; v += 3) {
    rot_vec(T, gr[v], gq[v]);                    /* scalar gradient */
    /* momentum: G' = m G m^T with G_ik = d m_i / d x_k */
    double G[2][2] = {{gr[v + 1][0], gr[v + 1][1]}, {gr[v + 2][0], gr[v + 2][1]}};
    double H[2][2];
    for (int a = 0; a < 2; a++)
      for (int b = 0; b < 2; b++) {
        double s = 0;
        for (int c = 0; c < 2; c++)
          for (int d = 0; d < 2; d++) s += T->m[a][c] * G[c][d] * T->m[b][d];
        H[a][b] = s;
      }
    gq[v + 1][0] = H[0][0]; gq[v + 1][1] = H[0][1];
    gq[v + 2][0] = H[1][0]; gq[v + 2][1] = H[1][1];
  }
}

/* ------------------------------------------------------------------------- */
/* reconstruction: P3 least squares, P1 candidates, WENO-Z combination (R5)   */
/* ------------------------------------------------------------------------- */
static double smoothness_p3(const orc_t *o, int j, const double a[NB]) {
  /* beta = sum_{1<=|alpha|<=3} |Omega|^{|alpha|-1} int (D^alpha p)^2, which in  */
  /* the scaled coordinates is the mean over the cell of (D_xi^alpha p)^2       */
  quad_init();
  double P[3][2];
  cell_vertices(o, j, P);
  double beta = 0;
  for (int q = 0; q < NQT; q++) {
    double x[2], xi[2];
    x[0] = P[0][0] + QT_A[q] * (P[1][0] - P[0][0]) + QT_B[q] * (P[2][0] - P[0][0]);
    x[1] = P[0][1] + QT_A[q] * (P[1][1] - P[0][1]) + QT_B[q] * (P[2][1] - P[0][1]);
    cell_to_xi(o, j, x, xi);
    double X = xi[0], Y = xi[1];
    double px = a[1] + a[3] * X + a[4] * Y + a[6] * X * X / 2 + a[7] * X * Y + a[8] * Y * Y / 2;
    double py = a[2] + a[4] * X + a[5] * Y + a[7] * X * X / 2 + a[8] * X * Y + a[9] * Y * Y / 2;
    double pxx = a[3] + a[6] * X + a[7] * Y;
    double pxy = a[4] + a[7] * X + a[8] * Y;
    double pyy = a[5] + a[8] * X + a[9] * Y;
    beta += QT_W[q] * (px * px + py * py + pxx * pxx + pxy * pxy + pyy * pyy);
  }
  beta += a[6] * a[6] + a[7] * a[7] + a[8] * a[8] + a[9] * a[9];
  return beta;
}

static void reconstruct(orc_t *o) {
  const double gh = o->gam_hi, gl = (1 - o->gam_hi) / 3;
  for (int j = 0; j < o->nt; j++) {
    image_t self = {j, aff_id()};
    double q0[NVAR], g0[NVAR][2];
    image_avg(o, &self, q0);
    image_grad(o, &self, g0);
    double h = o->hs[j];
    int n = o->navg[j];
    double qi[MAXAVG][NVAR], gf[3][NVAR][2];
    for (int s = 0; s < n; s++) image_avg(o, &o->avg_img[j * MAXAVG + s], qi[s]);
    for (int f = 0; f < 3; f++) image_grad(o, &o->face[IDX2(j, f)], gf[f]);
    for (int v = 0; v < NVAR; v++) {
      double rhs[MAXROWS];
      for (int c = 0; c < MAXROWS; c++) rhs[c] = 0;
      for (int s = 0; s < n; s++) rhs[s] = qi[s][v] - q0[v];
      rhs[9] = h * g0[v][0]; rhs[10] = h * g0[v][1];
      for (int f = 0; f < 3; f++) { rhs[11 + 2 * f] = h * gf[f][v][0]; rhs[12 + 2 * f] = h * gf[f][v][1]; }
      double a3[NB];
      a3[0] = q0[v];
      const double *Mj = &o->M[j * 9 * MAXROWS];
      for (int r = 0; r < 9; r++) {
        double s = 0;
        for (int c = 0; c < MAXROWS; c++) s += Mj[r * MAXROWS + c] * rhs[c];
        a3[r + 1] = s;
      }
      /* P1 candidates on {0, face f} */
      double b[3][2], beta[4];
      for (int f = 0; f < 3; f++) {
        /* face f's average row is stencil slot f (faces come first) */
        double r5[5] = {qi[f][v] - q0[v], h * g0[v][0], h * g0[v][1], h * gf[f][v][0], h * gf[f][v][1]};
        const double *N = &o->N1[(j * 3 + f) * 10];
        for (int d = 0; d < 2; d++) {
          double s = 0;
          for (int c = 0; c < 5; c++) s += N[d * 5 + c] * r5[c];
          b[f][d] = s;
        }
        beta[1 + f] = b[f][0] * b[f][0] + b[f][1] * b[f][1];
      }
      beta[0] = smoothness_p3(o, j, a3);
      /* WENO-Z weights */
      double tz = (fabs(beta[0] - beta[1]) + fabs(beta[0] - beta[2]) + fabs(beta[0] - beta[3])) / 3;
      double eps = o->weno_eps * o->area[j] * (1 + q0[v] * q0[v]);   /* R5: epsilon ~ h^2 */
      double gam[4] = {gh, gl, gl, gl}, w[4], ws = 0;
      for (int k = 0; k < 4; k++) {
        double r = tz / (beta[k] + eps);
        w[k] = gam[k] * (1 + r * r);
        ws += w[k];
      }
      for (int k = 0; k < 4; k++) w[k] /= ws;
      double dev = 0;
      for (int k = 0; k < 4; k++) dev = fmax(dev, fabs(w[k] / gam[k] - 1));
      o->wdev[j * NVAR + v] = dev;
      if (o->linear && o->linear[j]) {
        /* a cell the troubled-cell gate calls smooth: linear weights, so the */
        /* combination is the P3 polynomial itself (and the blend w is 1)     */
        for (int k = 0; k < 4; k++) w[k] = gam[k];
        o->wdev[j * NVAR + v] = 0;
      }
      /* R = (w_H/g_H) (P3 - sum g_m P1_m) + sum w_m P1_m, in the zero-mean basis */
      double *cf = &o->coef[(j * NVAR + v) * NB];
      double fac = w[0] / gh;
      cf[0] = q0[v];
      for (int k = 1; k < NB; k++) cf[k] = fac * a3[k];
      for (int f = 0; f < 3; f++) {
        cf[1] += (w[1 + f] - fac * gl) * b[f][0];
        cf[2] += (w[1 + f] - fac * gl) * b[f][1];
      }
      o->omegaH[j * NVAR + v] = w[0];
    }
  }
}

/* evaluate cell c's reconstruction at a point given in c's own frame */
static void eval_cell(const orc_t *o, int c, const double x[2], double val[NVAR], double grd[NVAR][2]) {
  double xi[2], m[NB], mx[NB], my[NB];
  cell_to_xi(o, c, x, xi);
  monomials(xi[0], xi[1], m);
  monomials_dx(xi[0], xi[1], mx);
  monomials_dy(xi[0], xi[1], my);
  const double *mean = &o->mean_m[c * NB];
  for (int v = 0; v < NVAR; v++) {
    const double *cf = &o->coef[(c * NVAR + v) * NB];
    double s = cf[0], sx = 0, sy = 0;
    for (int k = 1; k < NB; k++) {
      s += cf[k] * (m[k] - mean[k]);
      sx += cf[k] * mx[k];
      sy += cf[k] * my[k];
    }
    val[v] = s;
    grd[v][0] = sx / o->hs[c];
    grd[v][1] = sy / o->hs[c];
  }
}
/* evaluate an image at a point in the viewer's frame (values/gradients transformed) */
static void eval_image(const orc_t *o, const image_t *im, const double x[2], double val[NVAR], double grd[NVAR][2]) {
  double xc[2], v0[NVAR], g0[NVAR][2];
  aff_apply_inv(&im->T, x, xc);
  eval_cell(o, im->cell, xc, v0, g0);
  const aff_t *T = &im->T;
  for (int v = 0; v < NVAR; v += 3) {
    val[v] = v0[v];
    rot_vec(T, &v0[v + 1], &val[v + 1]);
    rot_vec(T, g0[v], grd[v]);
    double H[2][2];
    for (int a = 0; a < 2; a++)
      for (int b = 0; b < 2; b++) {
        double s = 0;
        for (int c = 0; c < 2; c++)
          for (int d = 0; d < 2; d++) s += T->m[a][c] * g0[v + 1 + c][d] * T->m[b][d];
        H[a][b] = s;
      }
    grd[v + 1][0] = H[0][0]; grd[v + 1][1] = H[0][1];
    grd[v + 2][0] = H[1][0]; grd[v + 2][1] = H[1][1];
  }
}

/* ------------------------------------------------------------------------- */
/* velocity-space polynomials and Maxwellian moments (Eqs. g-SWE, bgk-g-to-*) */
/* ------------------------------------------------------------------------- */
#define PD 8   /* moments up to order 7 */
#define PP 4   /* kernels are polynomials of degree <= 3 in u and in v */
typedef struct { double c[PP][PP]; } vpoly_t;   /* c[i][j]: coefficient of u^i v^j */

static void vp_zero(vpoly_t *p) { memset(p, 0, sizeof(*p)); }
static void vp_extent(const vpoly_t *p, int *mi, int *mj) {
  *mi = -1; *mj = -1;
  for (int i = 0; i < PP; i++)
    for (int j = 0; j < PP; j++)
      if (p->c[i][j] != 0) { if (i > *mi) *mi = i; if (j > *mj) *mj = j; }
}
/* set when a product would exceed the polynomial degree the kernels have: */
/* only non-finite coefficients (a non-physical interface state) do that;   */
/* orc_advance then stops with an error code instead of going on            */
static _Thread_local int vp_overflow = 0;
static void vp_mul(const vpoly_t *a, const vpoly_t *b, vpoly_t *out) {
  vpoly_t r;
  int ai, aj, bi, bj;
  vp_zero(&r);
  vp_extent(a, &ai, &aj);
  vp_extent(b, &bi, &bj);
  for (int i = 0; i <= ai; i++)
    for (int j = 0; j <= aj; j++) {
      if (a->c[i][j] == 0) continue;
      for (int k = 0; k <= bi; k++)
        for (int l = 0; l <= bj; l++) {
          if (i + k >= PP || j + l >= PP) { vp_overflow = 1; continue; }
          r.c[i + k][j + l] += a->c[i][j] * b->c[k][l];
        }
    }
  *out = r;
}
static void vp_axpy(double s, const vpoly_t *a, vpoly_t *y) {
  for (int i = 0; i < PP; i++)
    for (int j = 0; j < PP; j++) y->c[i][j] += s * a->c[i][j];
}
static void vp_lin(vpoly_t *p, double c0, double cu, double cv) {   /* c0 + cu u + cv v */
  vp_zero(p); p->c[0][0] = c0; p->c[1][0] = cu; p->c[0][1] = cv;
}

/* raw moments <u^k> of the normalised 1-D Maxwellian sqrt(lam/pi) e^{-lam (u-U)^2} */
/* over the full line (half=0), u>0 (half=+1) or u<0 (half=-1)                     */
void orc_raw_moments(double U, double lam, int half, int n, double *mu) {
  if (half == 0) { mu[0] = 1; if (n > 0) mu[1] = U; }
  else {
    double e = 0.5 * exp(-lam * U * U) / sqrt(M_PI * lam);
    if (half > 0) { mu[0] = 0.5 * erfc(-sqrt(lam) * U); if (n > 0) mu[1] = U * mu[0] + e; }
    else          { mu[0] = 0.5 * erfc(sqrt(lam) * U);  if (n > 0) mu[1] = U * mu[0] - e; }
  }
  for (int k = 0; k + 2 <= n; k++) mu[k + 2] = U * mu[k + 1] + (k + 1) / (2 * lam) * mu[k];
}

typedef struct { double h, U, V, lam; double mu[3][PD], nu[PD]; } maxw_t;

static maxw_t maxw(double h, double U, double V, double G) {
  maxw_t g;
  g.h = h; g.U = U; g.V = V; g.lam = 1 / (G * h);
  orc_raw_moments(U, g.lam, 0, PD - 1, g.mu[0]);
  orc_raw_moments(U, g.lam, +1, PD - 1, g.mu[1]);
  orc_raw_moments(U, g.lam, -1, PD - 1, g.mu[2]);
  orc_raw_moments(V, g.lam, 0, PD - 1, g.nu);
  return g;
}

/* int u^wi v^wj p(u,v) g du dv over the chosen u half-space,                 */
/* g = h (lam/pi) e^{-lam|u-U|^2}                                              */
static double vmoment_w(const vpoly_t *p, const maxw_t *g, int half, int wi, int wj) {
  const double *mu = g->mu[half == 0 ? 0 : (half > 0 ? 1 : 2)], *nu = g->nu;
  int mi, mj;
  vp_extent(p, &mi, &mj);
  double s = 0;
  for (int i = 0; i <= mi; i++)
    for (int j = 0; j <= mj; j++)
      if (p->c[i][j] != 0) s += p->c[i][j] * mu[i + wi] * nu[j + wj];
  return g->h * s;
}

/* slope term a.u of a Maxwellian base: a = d(ln g)/dx_k along n and t for the */
/* SWE Maxwellian with lam = 1/(G h) (reading R1): lam (dh/h)|u-U|^2 + 2 lam (u-U).dU */
static void slope_poly(const maxw_t *b, const double dn[3], const double dt[3], vpoly_t *out) {
  vpoly_t cu, cv, c2, t, an, at, u, v;
  vp_lin(&cu, -b->U, 1, 0);
  vp_lin(&cv, -b->V, 0, 1);
  vp_mul(&cu, &cu, &c2);
  vp_mul(&cv, &cv, &t);
  vp_axpy(1, &t, &c2);                               /* |u - U|^2 */
  const double *d[2] = {dn, dt};
  vpoly_t *a[2] = {&an, &at};
  for (int k = 0; k < 2; k++) {
    double dh = d[k][0];
    double dU = (d[k][1] - b->U * dh) / b->h;
    double dV = (d[k][2] - b->V * dh) / b->h;
    vp_zero(a[k]);
    vp_axpy(b->lam * dh / b->h, &c2, a[k]);
    vp_axpy(2 * b->lam * dU, &cu, a[k]);
    vp_axpy(2 * b->lam * dV, &cv, a[k]);
  }
  vp_lin(&u, 0, 1, 0);
  vp_lin(&v, 0, 0, 1);
  vpoly_t s1, s2;
  vp_mul(&an, &u, &s1);
  vp_mul(&at, &v, &s2);
  vp_zero(out);
  vp_axpy(1, &s1, out);
  vp_axpy(1, &s2, out);
}
/* force term. The paper writes -2 alpha_{k,m} lam gradPhi.(u-U) with moment-  */
/* dependent constants defined in an appendix outside the paper (reading R1):  */
/* we use -lam^2 |u-U|^2 gradPhi.(u-U), whose full-space moments with psi and  */
/* u psi equal those of the natural force -2 lam gradPhi.(u-U), and which at   */
/* rest cancels the slope term pointwise in u (every half-space moment).        */
static void force_poly(const maxw_t *b, double phin, double phit, vpoly_t *out) {
  vpoly_t cu, cv, c2, t, fc;
  vp_lin(&cu, -b->U, 1, 0);
  vp_lin(&cv, -b->V, 0, 1);
  vp_mul(&cu, &cu, &c2);
  vp_mul(&cv, &cv, &t);
  vp_axpy(1, &t, &c2);
  vp_lin(&fc, -phin * b->U - phit * b->V, phin, phit);
  vp_mul(&c2, &fc, out);
  for (int i = 0; i < PP; i++)
    for (int j = 0; j < PP; j++) out->c[i][j] *= -b->lam * b->lam;
}
/* time derivative kernel A of a Maxwellian from d/dt of (h, hU, hV) */
static void time_poly(const maxw_t *b, const double d[3], vpoly_t *out) {
  vpoly_t cu, cv, c2, t;
  vp_lin(&cu, -b->U, 1, 0);
  vp_lin(&cv, -b->V, 0, 1);
  vp_mul(&cu, &cu, &c2);
  vp_mul(&cv, &cv, &t);
  vp_axpy(1, &t, &c2);
  vp_zero(out);
  vp_axpy(b->lam * d[0] / b->h, &c2, out);
  vp_axpy(2 * b->lam * (d[1] - b->U * d[0]) / b->h, &cu, out);
  vp_axpy(2 * b->lam * (d[2] - b->V * d[0]) / b->h, &cv, out);
}

/* time integrals over [0, delta] of C1..C5 (coefficients under Eq. SWE-2nd-order) */
void orc_time_integrals(double tau, double delta, double q[5]) {
  double x = delta / tau;
  double em = -expm1(-x);         /* 1 - e^{-delta/tau} */
  double e = exp(-x);
  q[0] = delta - tau * em;
  q[1] = -tau * delta * (1 + e) + 2 * tau * tau * em;
  q[2] = 0.5 * delta * delta - tau * delta + tau * tau * em;
  q[3] = tau * em;
  q[4] = tau * delta * e - tau * tau * em;
}

/* side data of the interface problem in the local frame (x along n) */
typedef struct { double h, U, V; double dn[3], dt[3]; double phin, phit; } side_t;

/* moments of the five parts of f (Eq. SWE-2nd-order), weights psi and u psi */
static void gks_parts(const side_t *l, const side_t *r, double G, double Gp[5][6]) {
  maxw_t gl = maxw(l->h, l->U, l->V, G);
  maxw_t gr = maxw(r->h, r->U, r->V, G);
  /* weights: psi = (1, u, v) and u psi = (u, u^2, uv), as monomials u^wi v^wj */
  static const int WI[6] = {0, 1, 0, 1, 2, 1}, WJ[6] = {0, 0, 1, 0, 0, 1};
  vpoly_t one;
  vp_lin(&one, 1, 0, 0);
  /* W-bar: the t = 0 state at the interface (compatibility, Eq. bgk-g-to-W) */
  double wb[3];
  for (int k = 0; k < 3; k++) wb[k] = vmoment_w(&one, &gl, +1, WI[k], WJ[k]) + vmoment_w(&one, &gr, -1, WI[k], WJ[k]);
  maxw_t gb = maxw(wb[0], wb[1] / wb[0], wb[2] / wb[0], G);
  /* kernels */
  vpoly_t sbl, sbr, fbl, fbr, kbl, kbr, sl, sr, fl, fr, kl, kr;
  slope_poly(&gb, l->dn, l->dt, &sbl);
  slope_poly(&gb, r->dn, r->dt, &sbr);
  force_poly(&gb, l->phin, l->phit, &fbl);
  force_poly(&gb, r->phin, r->phit, &fbr);
  kbl = sbl; vp_axpy(1, &fbl, &kbl);
  kbr = sbr; vp_axpy(1, &fbr, &kbr);
  slope_poly(&gl, l->dn, l->dt, &sl);
  slope_poly(&gr, r->dn, r->dt, &sr);
  force_poly(&gl, l->phin, l->phit, &fl);
  force_poly(&gr, r->phin, r->phit, &fr);
  kl = sl; vp_axpy(1, &fl, &kl);
  kr = sr; vp_axpy(1, &fr, &kr);
  /* A-bar from compatibility: int psi (A-bar + a-bar.u + force) g-bar = 0 */
  double dA[3];
  for (int k = 0; k < 3; k++)
    dA[k] = -(vmoment_w(&kbl, &gb, +1, WI[k], WJ[k]) + vmoment_w(&kbr, &gb, -1, WI[k], WJ[k]));
  vpoly_t At;
  time_poly(&gb, dA, &At);
  for (int w = 0; w < 6; w++) {
    int a = WI[w], b = WJ[w];
    Gp[0][w] = vmoment_w(&one, &gb, 0, a, b);                                          /* C1: g-bar        */
    Gp[1][w] = vmoment_w(&kbl, &gb, +1, a, b) + vmoment_w(&kbr, &gb, -1, a, b);        /* C2: slopes+force */
    Gp[2][w] = vmoment_w(&At, &gb, 0, a, b);                                           /* C3: A-bar        */
    Gp[3][w] = vmoment_w(&one, &gl, +1, a, b) + vmoment_w(&one, &gr, -1, a, b);        /* C4: g^l, g^r     */
    Gp[4][w] = vmoment_w(&kl, &gl, +1, a, b) + vmoment_w(&kr, &gr, -1, a, b);          /* C5: transport    */
  }
}

/* time-integrated moments over [0, delta_i] for nd interval lengths:          */
/* W_int = int int psi f, F_int = int int u psi f                              */
static void gks_point_multi(const side_t *l, const side_t *r, double G, double tau, int nd,
                            const double *delta, double (*Wint)[3], double (*Fint)[3]) {
  double Gp[5][6], q[5];
  gks_parts(l, r, G, Gp);
  for (int i = 0; i < nd; i++) {
    orc_time_integrals(tau, delta[i], q);
    for (int k = 0; k < 3; k++) {
      double sw = 0, sf = 0;
      for (int p = 0; p < 5; p++) { sw += q[p] * Gp[p][k]; sf += q[p] * Gp[p][3 + k]; }
      Wint[i][k] = sw;
      Fint[i][k] = sf;
    }
  }
}
void orc_gks_point(const double *L /* side_t packed: h U V dn[3] dt[3] phin phit */,
                   const double *R, double G, double tau, double delta, double Wint[3], double Fint[3]) {
  side_t l, r;
  memcpy(&l, L, sizeof(side_t));
  memcpy(&r, R, sizeof(side_t));
  gks_point_multi(&l, &r, G, tau, 1, &delta, (double (*)[3])Wint, (double (*)[3])Fint);
}

/* ------------------------------------------------------------------------- */
/* one stage                                                                 */
/* ------------------------------------------------------------------------- */
static double cfl_dt(const orc_t *o) {
  double best = INFINITY;
  for (int j = 0; j < o->nt; j++) {
    const double *a = &o->avg[j * NVAR];
    double um = 0;
    for (int l = 0; l < 2; l++) {
      double h = a[3 * l], u = a[3 * l + 1] / h, v = a[3 * l + 2] / h;
      double s = sqrt(u * u + v * v) + sqrt(o->g * h);
      if (s > um) um = s;
    }
    double d = o->dX[j] / um;
    if (d < best) best = d;
  }
  return o->cfl * best;
}

/* S2O4 update (Eq. SWE-fully-discrete) */
double orc_s2o4(int stage, double Wn, double Ln, double Ltn, double Lt_half, double dt) {
  if (stage == 1) return Wn + 0.5 * dt * Ln + 0.125 * dt * dt * Ltn;
  return Wn + dt * Ln + dt * dt / 6 * Ltn + dt * dt / 3 * Lt_half;
}

/* local frame: n and t = (-n_y, n_x) */
static void to_local_side(const double val[NVAR], const double grd[NVAR][2], int layer_base,
                          const double n[2], side_t *s) {
  double t[2] = {-n[1], n[0]};
  int hb = layer_base, mb = layer_base + 1;
  s->h = val[hb];
  double mn = val[mb] * n[0] + val[mb + 1] * n[1];
  double mt = val[mb] * t[0] + val[mb + 1] * t[1];
  s->U = mn / s->h;
  s->V = mt / s->h;
  const double *dirs[2] = {n, t};
  double *outs[2] = {s->dn, s->dt};
  for (int k = 0; k < 2; k++) {
    const double *e = dirs[k];
    double dh = grd[hb][0] * e[0] + grd[hb][1] * e[1];
    double dmx = grd[mb][0] * e[0] + grd[mb][1] * e[1];
    double dmy = grd[mb + 1][0] * e[0] + grd[mb + 1][1] * e[1];
    outs[k][0] = dh;
    outs[k][1] = dmx * n[0] + dmy * n[1];
    outs[k][2] = dmx * t[0] + dmy * t[1];
  }
}

/* Positivity option (not in the paper, which states no limiter; off by      */
/* default, pos_floor = 0). After the reconstruction, a layer whose depth at  */
/* one of the cell's six edge Gauss points falls below pos_floor times the    */
/* cell's average depth has its depth and both discharge polynomials pulled  */
/* toward their cell averages by one factor theta, so that the least point    */
/* depth meets the floor (averages unchanged, so conservation is untouched); */
/* for the lower layer the depth is eta1 - B, so the bottom's linear part is  */
/* kept out of the scaling.                                                   */
static void positivity_scale(orc_t *o) {
  if (!o->pos_scaled) o->pos_scaled = calloc(2 * (size_t)o->nt, 1);
  for (int j = 0; j < o->nt; j++) {
    o->pos_scaled[2 * j] = o->pos_scaled[2 * j + 1] = 0;
    double hmin[2] = {INFINITY, INFINITY};   /* [0] lower layer h1, [1] upper layer h2 */
    for (int f = 0; f < 3; f++) {
      const edge_t *E = &o->edge[o->face_edge[IDX2(j, f)]];
      for (int q = 0; q < 2; q++) {
        double x[2], val[NVAR], grd[NVAR][2];
        if (o->face_side[IDX2(j, f)] > 0) { x[0] = E->xq[q][0]; x[1] = E->xq[q][1]; }
        else aff_apply_inv(&E->R.T, E->xq[q], x);
        eval_cell(o, j, x, val, grd);
        hmin[0] = fmin(hmin[0], val[3] - E->bq[q]);
        hmin[1] = fmin(hmin[1], val[0]);
      }
    }
    for (int l = 0; l < 2; l++) {
      const int v = l == 0 ? 3 : 0;
      const double hbar = o->coef[(j * NVAR + v) * NB] - (l == 0 ? o->bmean[j] : 0.0);
      const double fl = o->pos_floor * hbar;
      /* a layer whose point depths dip below half its average has its point */
      /* velocities bounded at its edges (the discharge slope of a steep jump */
      /* would otherwise meet a small depth)                                 */
      if (hmin[l] < 0.5 * hbar) o->pos_scaled[2 * j + l] = 1;
      if (hmin[l] >= fl) continue;
      const double th = fmax(0.0, (hbar - fl) / (hbar - hmin[l]));
      for (int m = 0; m < 3; m++) {
        double *cf = &o->coef[(j * NVAR + v + m) * NB];
        for (int k = 1; k < NB; k++) cf[k] *= th;
      }
      if (l == 0) {   /* eta1 = h1 + B: B's linear part stays */
        o->coef[(j * NVAR + 3) * NB + 1] += (1 - th) * o->hs[j] * o->bgrad[2 * j];
        o->coef[(j * NVAR + 3) * NB + 2] += (1 - th) * o->hs[j] * o->bgrad[2 * j + 1];
      }
    }
  }
}

static void stage(orc_t *o, int st) {
  const double dt = o->dt;
  /* the fit interval (reading R20): both stages fit the value and time     */
  /* derivative at their start from the time integrals over dt and dt/2   */
  /* (the S2O4 construction of Sec. 3.3 repeated from the intermediate    */
  /* state)                                                                */
  const double delta = dt;
  const double G = o->g;
  reconstruct(o);
  if (o->pos_floor > 0) positivity_scale(o);
  /* interface values at each Gauss point, both sides (R3, R7) */
  int ne = o->ne;
  double (*vl)[2][NVAR] = malloc(sizeof(double) * ne * 2 * NVAR);
  double (*vr)[2][NVAR] = malloc(sizeof(double) * ne * 2 * NVAR);
  double (*gl)[2][NVAR][2] = malloc(sizeof(double) * ne * 2 * NVAR * 2);
  double (*gr)[2][NVAR][2] = malloc(sizeof(double) * ne * 2 * NVAR * 2);
  for (int e = 0; e < ne; e++) {
    edge_t *E = &o->edge[e];
    image_t selfL = {E->L, aff_id()};
    double hc1 = 0, hc2 = 0;
    for (int q = 0; q < 2; q++) {
      eval_image(o, &selfL, E->xq[q], vl[e][q], gl[e][q]);
      eval_image(o, &E->R, E->xq[q], vr[e][q], gr[e][q]);
      /* water level -> depth: h1 = eta1 - B, grad h1 = grad eta1 - grad B */
      double gbL[2] = {o->bgrad[2 * E->L], o->bgrad[2 * E->L + 1]}, gbR[2];
      rot_vec(&E->R.T, &o->bgrad[2 * E->R.cell], gbR);
      vl[e][q][3] -= E->bq[q];
      vr[e][q][3] -= E->bq[q];
      for (int d = 0; d < 2; d++) { gl[e][q][3][d] -= gbL[d]; gr[e][q][3][d] -= gbR[d]; }
      /* h-hat = xi h^l + (1 - xi) h^r, xi = erfc((U^l + U^r)/2)/2 per layer */
      double unl1 = (vl[e][q][4] * E->n[0] + vl[e][q][5] * E->n[1]) / vl[e][q][3];
      double unr1 = (vr[e][q][4] * E->n[0] + vr[e][q][5] * E->n[1]) / vr[e][q][3];
      double unl2 = (vl[e][q][1] * E->n[0] + vl[e][q][2] * E->n[1]) / vl[e][q][0];
      double unr2 = (vr[e][q][1] * E->n[0] + vr[e][q][2] * E->n[1]) / vr[e][q][0];
      double xi1 = 0.5 * erfc(0.5 * (unl1 + unr1));
      double xi2 = 0.5 * erfc(0.5 * (unl2 + unr2));
      hc1 += 0.5 * (xi1 * vl[e][q][3] + (1 - xi1) * vr[e][q][3]);
      hc2 += 0.5 * (xi2 * vl[e][q][0] + (1 - xi2) * vr[e][q][0]);
    }
    o->hc[2 * e] = hc1;
    o->hc[2 * e + 1] = hc2;
  }
  /* per cell: the plane through the three edge-centre values (Sec. 2.3) */
  for (int j = 0; j < o->nt; j++) {
    double X[3][2], V1[3], V2[3];
    for (int f = 0; f < 3; f++) {
      int e = o->face_edge[IDX2(j, f)];
      edge_t *E = &o->edge[e];
      if (o->face_side[IDX2(j, f)] > 0) { X[f][0] = E->mid[0]; X[f][1] = E->mid[1]; }
      else aff_apply_inv(&E->R.T, E->mid, X[f]);
      V1[f] = o->hc[2 * e];
      V2[f] = o->hc[2 * e + 1];
    }
    double a11 = X[1][0] - X[0][0], a12 = X[1][1] - X[0][1];
    double a21 = X[2][0] - X[0][0], a22 = X[2][1] - X[0][1];
    double det = a11 * a22 - a12 * a21;
    double r1 = V1[1] - V1[0], r2 = V1[2] - V1[0];
    o->plane[4 * j + 0] = (r1 * a22 - r2 * a12) / det;
    o->plane[4 * j + 1] = (a11 * r2 - a21 * r1) / det;
    r1 = V2[1] - V2[0]; r2 = V2[2] - V2[0];
    o->plane[4 * j + 2] = (r1 * a22 - r2 * a12) / det;
    o->plane[4 * j + 3] = (a11 * r2 - a21 * r1) / det;
  }
  /* gas-kinetic interface solution per Gauss point and layer */
  for (int e = 0; e < ne; e++) {
    edge_t *E = &o->edge[e];
    const double *n = E->n;
    double t[2] = {-n[1], n[0]};
    /* side planes and weights (R6): w = clamp(min(omega_H^L, omega_H^R)/gamma_H, 0, 1) */
    double plL[4], plR[4];
    for (int k = 0; k < 4; k++) plL[k] = o->plane[4 * E->L + k];
    rot_vec(&E->R.T, &o->plane[4 * E->R.cell], &plR[0]);
    rot_vec(&E->R.T, &o->plane[4 * E->R.cell + 2], &plR[2]);
    double w1 = fmin(o->omegaH[E->L * NVAR + 3], o->omegaH[E->R.cell * NVAR + 3]) / o->gam_hi;
    double w2 = fmin(o->omegaH[E->L * NVAR + 0], o->omegaH[E->R.cell * NVAR + 0]) / o->gam_hi;
    w1 = fmax(0, fmin(1, w1));
    w2 = fmax(0, fmin(1, w2));
    double gbL[2] = {o->bgrad[2 * E->L], o->bgrad[2 * E->L + 1]}, gbR[2];
    rot_vec(&E->R.T, &o->bgrad[2 * E->R.cell], gbR);
    for (int q = 0; q < 2; q++) {
      double *V[2] = {vl[e][q], vr[e][q]};
      double (*Gd[2])[2] = {gl[e][q], gr[e][q]};
      double *pl[2] = {plL, plR};
      double *gb[2] = {gbL, gbR};
      double out[4][NVAR];   /* F, Ft, W, Wt */
      for (int layer = 0; layer < 2; layer++) {
        /* layer 0 of the loop: upper layer 2 (vars 0..2); layer 1: lower layer 1 (vars 3..5) */
        int base = layer == 0 ? 0 : 3;
        side_t s[2];
        for (int sd = 0; sd < 2; sd++) {
          to_local_side(V[sd], Gd[sd], base, n, &s[sd]);
          const int own_cell = sd == 0 ? E->L : E->R.cell, lay = base == 3 ? 0 : 1;
          if (o->pos_floor > 0 && o->pos_scaled[2 * own_cell + lay]) {
            /* positivity option, on a side whose depth polynomial was        */
            /* scaled: the point velocity kept within the two cells' average  */
            /* velocities of the layer (R's seen through its image), so a    */
            /* depth pulled up toward the floor cannot carry the discharge   */
            /* slope of a jump into a spurious vacuum                         */
            const double hL = o->avg[E->L * NVAR + base], hR = o->avg[E->R.cell * NVAR + base];
            const double uL[2] = {o->avg[E->L * NVAR + base + 1] / hL, o->avg[E->L * NVAR + base + 2] / hL};
            const double uR0[2] = {o->avg[E->R.cell * NVAR + base + 1] / hR,
                                   o->avg[E->R.cell * NVAR + base + 2] / hR};
            double uR[2];
            rot_vec(&E->R.T, uR0, uR);
            const double nl = uL[0] * n[0] + uL[1] * n[1], nr = uR[0] * n[0] + uR[1] * n[1];
            const double tl = uL[0] * t[0] + uL[1] * t[1], tr = uR[0] * t[0] + uR[1] * t[1];
            s[sd].U = fmin(fmax(s[sd].U, fmin(nl, nr)), fmax(nl, nr));
            s[sd].V = fmin(fmax(s[sd].V, fmin(tl, tr)), fmax(tl, tr));
          }
          /* acceleration (Eq. bgk-phi, Sec. 2.3) with the blended derivative of */
          /* the other layer's depth                                              */
          double ht[2], ph[2];
          if (base == 0) {   /* upper layer: grad Phi_2 = -G grad B - G grad h1~ */
            for (int d = 0; d < 2; d++) {
              ht[d] = w1 * Gd[sd][3][d] + (1 - w1) * pl[sd][d];
              ph[d] = -G * gb[sd][d] - G * ht[d];
            }
          } else {           /* lower layer: grad Phi_1 = -G grad B - chi G grad h2~ */
            for (int d = 0; d < 2; d++) {
              ht[d] = w2 * Gd[sd][0][d] + (1 - w2) * pl[sd][2 + d];
              ph[d] = -G * gb[sd][d] - o->chi * G * ht[d];
            }
          }
          s[sd].phin = ph[0] * n[0] + ph[1] * n[1];
          s[sd].phit = ph[0] * t[0] + ph[1] * t[1];
        }
        /* collision time (Sec. 4): tau = eps dt + eps_num |(hl^2-hr^2)/(hl^2+hr^2)| dt */
        double hl2 = s[0].h * s[0].h, hr2 = s[1].h * s[1].h;
        double tau = o->eps * dt + o->eps_num * fabs((hl2 - hr2) / (hl2 + hr2)) * dt;
        double Wi[2][3], Fi[2][3], dl[2] = {delta, 0.5 * delta};
        gks_point_multi(&s[0], &s[1], G, tau, 2, dl, Wi, Fi);
        double *W1 = Wi[0], *W2 = Wi[1], *F1 = Fi[0], *F2 = Fi[1];
        /* value and time derivative at the stage start from the two integrals */
        double Fl[3], Ftl[3], Wl[3], Wtl[3];
        for (int k = 0; k < 3; k++) {
          Fl[k] = (4 * F2[k] - F1[k]) / delta;
          Ftl[k] = 4 * (F1[k] - 2 * F2[k]) / (delta * delta);
          Wl[k] = (4 * W2[k] - W1[k]) / delta;
          Wtl[k] = 4 * (W1[k] - 2 * W2[k]) / (delta * delta);
        }
        double *loc[4] = {Fl, Ftl, Wl, Wtl};
        for (int k = 0; k < 4; k++) {
          out[k][base] = loc[k][0];
          out[k][base + 1] = loc[k][1] * n[0] + loc[k][2] * t[0];
          out[k][base + 2] = loc[k][1] * n[1] + loc[k][2] * t[1];
        }
      }
      for (int v = 0; v < NVAR; v++) {
        o->eF[(e * 2 + q) * NVAR + v] = out[0][v];
        o->eFt[(e * 2 + q) * NVAR + v] = out[1][v];
        o->eW[(e * 2 + q) * NVAR + v] = out[2][v];
        o->eWt[(e * 2 + q) * NVAR + v] = out[3][v];
      }
    }
  }
  free(gl); free(gr);
  if (st == 1) memcpy(o->eWn, o->eW, sizeof(double) * ne * 2 * NVAR);
  /* cell residuals and update */
  double *newavg = malloc(sizeof(double) * o->nt * NVAR);
  double *newgrad = malloc(sizeof(double) * o->nt * NVAR * 2);
  for (int j = 0; j < o->nt; j++) {
    double A = o->area[j];
    double LF[NVAR] = {0}, LFt[NVAR] = {0};
    double mWt[NVAR] = {0};                          /* mean over the 6 Gauss points */
    double GGt[NVAR][2] = {{0}}, GGn[NVAR][2] = {{0}};
    /* the cell's own reconstruction at its six Gauss points (reading R16):   */
    /* the mean of h over them and their Gauss-theorem gradient               */
    double mO[NVAR] = {0}, GO[NVAR][2] = {{0}};
    for (int f = 0; f < 3; f++) {
      int e = o->face_edge[IDX2(j, f)];
      double sg = o->face_side[IDX2(j, f)];
      edge_t *E = &o->edge[e];
      for (int q = 0; q < 2; q++) {
        for (int v = 0; v < NVAR; v++) {
          double F = o->eF[(e * 2 + q) * NVAR + v], Ft = o->eFt[(e * 2 + q) * NVAR + v];
          double Wt = o->eWt[(e * 2 + q) * NVAR + v];
          double Wn = o->eWn[(e * 2 + q) * NVAR + v];
          double Wo = sg > 0 ? vl[e][q][v] : vr[e][q][v];   /* this cell's side */
          LF[v] -= sg * E->len * 0.5 * F / A;          /* Eq. SWE-semi-flux */
          LFt[v] -= sg * E->len * 0.5 * Ft / A;
          mO[v] += Wo / 6;
          mWt[v] += Wt / 6;
          /* interface value at the stage end (Eq. S2O3) */
          double Wend = (st == 1) ? Wn + 0.5 * dt * Wt : Wn + dt * Wt;
          for (int d = 0; d < 2; d++) {
            GO[v][d] += sg * E->len * E->n[d] * 0.5 * Wo / A;     /* Gauss theorem (Eq. slope-1) */
            GGt[v][d] += sg * E->len * E->n[d] * 0.5 * Wt / A;
            GGn[v][d] += sg * E->len * E->n[d] * 0.5 * Wend / A;
          }
        }
      }
    }
    const double *a = &o->avg[j * NVAR];
    const double *gB = &o->bgrad[2 * j];
    double L[NVAR], Lt[NVAR];
    for (int v = 0; v < NVAR; v++) { L[v] = LF[v]; Lt[v] = LFt[v]; }
    /* bottom source L^S1 = h_j (0, -G B_x, -G B_y) and its time derivative */
    for (int l = 0; l < 2; l++) {
      int b = 3 * l;
      for (int d = 0; d < 2; d++) {
        L[b + 1 + d] += -G * a[b] * gB[d];
        Lt[b + 1 + d] += -G * LF[b] * gB[d];
      }
    }
    /* interlayer source L^S2 (Eq. SWE-source-discretization): the point     */
    /* values are the cell's own reconstruction at its six Gauss points      */
    /* (reading R16); the time derivative by the product rule with the       */
    /* interface solution's time derivatives W_t (reading R4)                */
    for (int d = 0; d < 2; d++) {
      /* upper: -G mean(h2) * GaussGrad(h1) */
      L[1 + d] += -G * mO[0] * GO[3][d];
      Lt[1 + d] += -G * (mWt[0] * GO[3][d] + mO[0] * GGt[3][d]);
      /* lower: -chi G mean(h1) * GaussGrad(h2) */
      L[4 + d] += -o->chi * G * mO[3] * GO[0][d];
      Lt[4 + d] += -o->chi * G * (mWt[3] * GO[0][d] + mO[3] * GGt[0][d]);
    }
    for (int v = 0; v < NVAR; v++) {
      if (st == 1) {
        o->Wn[j * NVAR + v] = a[v];
        o->Ln[j * NVAR + v] = L[v];
        o->Ltn[j * NVAR + v] = Lt[v];
        newavg[j * NVAR + v] = orc_s2o4(1, a[v], L[v], Lt[v], 0, dt);
      } else {
        newavg[j * NVAR + v] = orc_s2o4(2, o->Wn[j * NVAR + v], o->Ln[j * NVAR + v], o->Ltn[j * NVAR + v], Lt[v], dt);
      }
      newgrad[(j * NVAR + v) * 2] = GGn[v][0];
      newgrad[(j * NVAR + v) * 2 + 1] = GGn[v][1];
    }
  }
  memcpy(o->avg, newavg, sizeof(double) * o->nt * NVAR);
  memcpy(o->grad, newgrad, sizeof(double) * o->nt * NVAR * 2);
  free(newavg); free(newgrad);
  free(vl); free(vr);
}

/* ------------------------------------------------------------------------- */
/* public (ctypes) interface                                                 */
/* ------------------------------------------------------------------------- */
orc_t *orc_create(int nv, const double *xy, int nt, const int *tri, const signed char *tri_bc,
                  double px, double py, const double *bvert,
                  double g, double chi, double cfl, double eps, double eps_num,
                  double gam_hi, double weno_eps, int *status) {
  orc_t *o = calloc(1, sizeof(orc_t));
  o->nv = nv; o->nt = nt;
  o->xy = malloc(sizeof(double) * 2 * nv); memcpy(o->xy, xy, sizeof(double) * 2 * nv);
  o->tri = malloc(sizeof(int) * 3 * nt); memcpy(o->tri, tri, sizeof(int) * 3 * nt);
  o->tri_bc = malloc(3 * nt);
  if (tri_bc) memcpy(o->tri_bc, tri_bc, 3 * nt); else memset(o->tri_bc, BC_WALL, 3 * nt);
  o->period[0] = px; o->period[1] = py;
  o->bvert = calloc(nv, sizeof(double));
  if (bvert) memcpy(o->bvert, bvert, sizeof(double) * nv);
  o->g = g; o->chi = chi; o->cfl = cfl; o->eps = eps; o->eps_num = eps_num;
  o->gam_hi = gam_hi; o->weno_eps = weno_eps;
  o->area = malloc(sizeof(double) * nt); o->cx = malloc(sizeof(double) * nt); o->cy = malloc(sizeof(double) * nt);
  o->hs = malloc(sizeof(double) * nt); o->dX = malloc(sizeof(double) * nt);
  o->bmean = malloc(sizeof(double) * nt); o->bgrad = malloc(sizeof(double) * 2 * nt);
  o->mean_m = malloc(sizeof(double) * NB * nt);
  o->face = malloc(sizeof(image_t) * 3 * nt);
  o->face_edge = malloc(sizeof(int) * 3 * nt); o->face_side = malloc(sizeof(int) * 3 * nt);
  o->navg = malloc(sizeof(int) * nt);
  o->avg_img = malloc(sizeof(image_t) * MAXAVG * nt);
  o->M = malloc(sizeof(double) * 9 * MAXROWS * nt);
  o->N1 = malloc(sizeof(double) * 30 * nt);
  int st = build_mesh(o);
  if (!st) { build_bathymetry(o); st = build_operators(o); }
  *status = st;
  int ne = o->ne;
  o->avg = calloc(NVAR * nt, sizeof(double));
  o->grad = calloc(2 * NVAR * nt, sizeof(double));
  o->coef = calloc(NB * NVAR * nt, sizeof(double));
  o->omegaH = calloc(NVAR * nt, sizeof(double));
  o->wdev = calloc(NVAR * nt, sizeof(double));
  o->hc = calloc(2 * ne, sizeof(double));
  o->plane = calloc(4 * nt, sizeof(double));
  o->eF = calloc(2 * NVAR * ne, sizeof(double)); o->eFt = calloc(2 * NVAR * ne, sizeof(double));
  o->eW = calloc(2 * NVAR * ne, sizeof(double)); o->eWt = calloc(2 * NVAR * ne, sizeof(double));
  o->eWn = calloc(2 * NVAR * ne, sizeof(double));
  o->Wn = calloc(NVAR * nt, sizeof(double)); o->Ln = calloc(NVAR * nt, sizeof(double));
  o->Ltn = calloc(NVAR * nt, sizeof(double));
  return o;
}

void orc_destroy(orc_t *o) {
  if (o) free(o->pos_scaled);
  if (!o) return;
  void *ptrs[] = {o->xy, o->tri, o->tri_bc, o->bvert, o->area, o->cx, o->cy, o->hs, o->dX, o->bmean,
                  o->bgrad, o->mean_m, o->face, o->face_edge, o->face_side, o->navg, o->avg_img, o->M,
                  o->N1, o->edge, o->avg, o->grad, o->coef, o->omegaH, o->hc, o->plane, o->eF, o->eFt,
                  o->eW, o->eWt, o->eWn, o->Wn, o->Ln, o->Ltn, o->wdev, o->linear};
  for (size_t i = 0; i < sizeof(ptrs) / sizeof(ptrs[0]); i++) free(ptrs[i]);
  free(o);
}

int orc_num_edges(const orc_t *o) { return o->ne; }

/* state in variable-major arrays: avg[v*nt + j], grad[(v*2+d)*nt + j] */
void orc_set_state(orc_t *o, const double *avg, const double *grad) {
  for (int j = 0; j < o->nt; j++)
    for (int v = 0; v < NVAR; v++) {
      o->avg[j * NVAR + v] = avg[v * o->nt + j];
      for (int d = 0; d < 2; d++) o->grad[(j * NVAR + v) * 2 + d] = grad ? grad[(v * 2 + d) * o->nt + j] : 0;
    }
  o->t = 0; o->phase = 0; o->stages_done = 0;
}
void orc_get_state(const orc_t *o, double *avg, double *grad) {
  for (int j = 0; j < o->nt; j++)
    for (int v = 0; v < NVAR; v++) {
      avg[v * o->nt + j] = o->avg[j * NVAR + v];
      if (grad)
        for (int d = 0; d < 2; d++) grad[(v * 2 + d) * o->nt + j] = o->grad[(j * NVAR + v) * 2 + d];
    }
}

/* advance by up to n_stages stages; with t_end > 0 the step is shortened to  */
/* land on t_end and no further step starts once t_end is reached             */
int orc_advance(orc_t *o, int n_stages, double t_end, double *t_out) {
  for (int s = 0; s < n_stages; s++) {
    if (o->phase == 0) {
      double dt = cfl_dt(o);
      if (t_end > 0) {
        double rem = t_end - o->t;
        if (rem <= 1e-12 * fmax(1.0, fabs(t_end))) break;
        if (dt > rem) dt = rem;
      }
      if (!(dt > 0) || !isfinite(dt)) return -10;
      o->dt = dt;
      stage(o, 1);
      o->phase = 1;
    } else {
      stage(o, 2);
      o->t += o->dt;
      o->phase = 0;
    }
    o->stages_done++;
    if (vp_overflow) {
      vp_overflow = 0;
      return -11;   /* a non-finite interface state in this stage */
    }
  }
  if (t_out) *t_out = o->t;
  return 0;
}

double orc_last_dt(const orc_t *o) { return o->dt; }
double orc_time(const orc_t *o) { return o->t; }
long long orc_stages_done(const orc_t *o) { return o->stages_done; }

/* per-layer mass sum |Omega_j| h_j (layer 1 lower, layer 2 upper) */
void orc_mass(const orc_t *o, double mass[2]) {
  mass[0] = mass[1] = 0;
  for (int j = 0; j < o->nt; j++) {
    mass[0] += o->area[j] * o->avg[j * NVAR + 3];
    mass[1] += o->area[j] * o->avg[j * NVAR + 0];
  }
}
void orc_cell_geometry(const orc_t *o, double *area, double *cx, double *cy) {
  for (int j = 0; j < o->nt; j++) { area[j] = o->area[j]; cx[j] = o->cx[j]; cy[j] = o->cy[j]; }
}

/* pins: reconstruct from the current state, then evaluate cell c's polynomials */
void orc_reconstruct(orc_t *o) { reconstruct(o); }
/* the positivity option (not in the paper): depth floor as a fraction of the */
/* cell's average depth, 0 = off (the default)                                */
void orc_set_positivity(orc_t *o, double floor_fraction) { o->pos_floor = floor_fraction; }
/* the option's scaling alone, on the current reconstruction (pins) */
void orc_positivity_scale(orc_t *o) { if (o->pos_floor > 0) positivity_scale(o); }
void orc_eval(const orc_t *o, int c, double x, double y, double *val6, double *grad12) {
  double p[2] = {x, y}, v[NVAR], g[NVAR][2];
  eval_cell(o, c, p, v, g);
  for (int k = 0; k < NVAR; k++) { val6[k] = v[k]; grad12[2 * k] = g[k][0]; grad12[2 * k + 1] = g[k][1]; }
}
void orc_omega(const orc_t *o, double *om /* nt*6 */) { memcpy(om, o->omegaH, sizeof(double) * o->nt * NVAR); }

/* ---- troubled-cell gate (an addition to the paper's scheme) -------------- */
/* Largest departure of the four WENO weights from the linear ones, per      */
/* (cell, variable), from the last reconstruction.                           */
void orc_weight_departure(const orc_t *o, double *out /* nt*6 */) {
  memcpy(out, o->wdev, sizeof(double) * o->nt * NVAR);
}
/* Cells with mask[j] = 1 take the linear weights in every later            */
/* reconstruction; NULL removes the mask.                                    */
void orc_set_linear_mask(orc_t *o, const unsigned char *mask) {
  free(o->linear);
  o->linear = NULL;
  if (mask) {
    o->linear = malloc(o->nt);
    memcpy(o->linear, mask, o->nt);
  }
}
/* Gate inputs of every cell at the current state: for eta1 (columns 0-11)   */
/* and h2 (columns 12-23), over the cell and its three face neighbours       */
/* (face k is the edge from vertex k to vertex k+1), the deviation of the    */
/* average from the mean of the four and the size-scaled gradient hs * grad, */
/* all divided by sqrt(sum of their squares + weno_eps |Omega| (1 + q0^2)).  */
void orc_gate_features(const orc_t *o, double *X /* nt*24 */) {
  const int var[2] = {3, 0};
  for (int j = 0; j < o->nt; j++) {
    image_t self = {j, aff_id()};
    double q[4][NVAR], g[4][NVAR][2];
    image_avg(o, &self, q[0]);
    image_grad(o, &self, g[0]);
    for (int f = 0; f < 3; f++) {
      image_avg(o, &o->face[IDX2(j, f)], q[1 + f]);
      image_grad(o, &o->face[IDX2(j, f)], g[1 + f]);
    }
    for (int s = 0; s < 2; s++) {
      int v = var[s];
      double mean = (q[0][v] + q[1][v] + q[2][v] + q[3][v]) / 4, raw[12], ss = 0;
      for (int m = 0; m < 4; m++) {
        raw[3 * m] = q[m][v] - mean;
        raw[3 * m + 1] = o->hs[j] * g[m][v][0];
        raw[3 * m + 2] = o->hs[j] * g[m][v][1];
      }
      for (int k = 0; k < 12; k++) ss += raw[k] * raw[k];
      ss += o->weno_eps * o->area[j] * (1 + q[0][v] * q[0][v]);
      for (int k = 0; k < 12; k++) X[j * 24 + 12 * s + k] = raw[k] / sqrt(ss);
    }
  }
}
int orc_stencil_size(const orc_t *o, int c) { return o->navg[c]; }

/* Gauss points of every edge (L's frame) and the Gauss-theorem gradient of  */
/* point data (Eq. slope-1) for the exactness pin                            */
void orc_edge_points(const orc_t *o, double *xq /* ne*2*2 */, int *LR /* ne*2 */) {
  for (int e = 0; e < o->ne; e++) {
    for (int q = 0; q < 2; q++) { xq[(e * 2 + q) * 2] = o->edge[e].xq[q][0]; xq[(e * 2 + q) * 2 + 1] = o->edge[e].xq[q][1]; }
    LR[2 * e] = o->edge[e].L;
    LR[2 * e + 1] = o->edge[e].bc == BC_WALL ? -1 : o->edge[e].R.cell;
  }
}
void orc_gauss_gradient(const orc_t *o, const double *pv /* ne*2 */, double *g /* nt*2 */) {
  for (int j = 0; j < o->nt; j++) {
    double s[2] = {0, 0};
    for (int f = 0; f < 3; f++) {
      int e = o->face_edge[IDX2(j, f)];
      double sg = o->face_side[IDX2(j, f)];
      for (int q = 0; q < 2; q++)
        for (int d = 0; d < 2; d++) s[d] += sg * o->edge[e].len * o->edge[e].n[d] * 0.5 * pv[2 * e + q];
    }
    g[2 * j] = s[0] / o->area[j];
    g[2 * j + 1] = s[1] / o->area[j];
  }
}
/* edge-centre blended levels of the last stage (Sec. 2.3), formed from the  */
/* stage-start reconstruction: per edge, the lower layer's depth h1-hat and  */
/* the upper layer's h2-hat                                                  */
void orc_blend_levels(const orc_t *o, double *hc /* ne*2 */) {
  memcpy(hc, o->hc, sizeof(double) * 2 * (size_t)o->ne);
}
/* per cell, the gradients of the planes through its three edge-centre      */
/* blended levels of the last stage (Sec. 2.3): d/dx, d/dy of h1-hat, h2-hat */
void orc_plane_gradients(const orc_t *o, double *pg /* nt*4 */) {
  memcpy(pg, o->plane, sizeof(double) * 4 * (size_t)o->nt);
}
/* interface data of the last stage: per edge per Gauss point, 6 values each */
void orc_edge_outputs(const orc_t *o, double *F, double *Ft, double *W, double *Wt) {
  size_t n = (size_t)o->ne * 2 * NVAR;
  if (F) memcpy(F, o->eF, n * sizeof(double));
  if (Ft) memcpy(Ft, o->eFt, n * sizeof(double));
  if (W) memcpy(W, o->eW, n * sizeof(double));
  if (Wt) memcpy(Wt, o->eWt, n * sizeof(double));
}
