// Host-side mesh preparation (FP64): cell renumbering along a Morton curve,
// edges with periodic matching and wall mirrors, the compact stencil of
// Eq. Recons-stencil, the least-squares operator of Eq. Recons-system, the
// P1 sub-stencil operators and smoothness form of the WENO reading, the plane
// operator of the interlayer force model (Sec. 2.3) and the edge geometry
// with 2-point Gauss quadrature (Eq. SWE-semi-flux).
#include "prep.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <thread>
#include <unordered_map>

namespace gks2l {
namespace {

// ---------------------------------------------------------------- isometries
struct Iso {
  double a, b, c, d, tx, ty;  // x' = [a b; c d] x + t
};
Iso iso_id() { return {1, 0, 0, 1, 0, 0}; }
Iso iso_shift(double sx, double sy) { return {1, 0, 0, 1, sx, sy}; }
// reflection across the line through (px, py) with unit normal (nx, ny)
Iso iso_mirror(double px, double py, double nx, double ny) {
  double pn = px * nx + py * ny;
  return {1 - 2 * nx * nx, -2 * nx * ny, -2 * nx * ny, 1 - 2 * ny * ny, 2 * pn * nx, 2 * pn * ny};
}
Iso iso_mul(const Iso &A, const Iso &B) {  // A o B
  return {A.a * B.a + A.b * B.c, A.a * B.b + A.b * B.d, A.c * B.a + A.d * B.c, A.c * B.b + A.d * B.d,
          A.a * B.tx + A.b * B.ty + A.tx, A.c * B.tx + A.d * B.ty + A.ty};
}
void iso_apply(const Iso &T, double x, double y, double &ox, double &oy) {
  ox = T.a * x + T.b * y + T.tx;
  oy = T.c * x + T.d * y + T.ty;
}
void iso_apply_inv(const Iso &T, double x, double y, double &ox, double &oy) {
  double dx = x - T.tx, dy = y - T.ty;  // orthogonal: inverse is the transpose
  ox = T.a * dx + T.c * dy;
  oy = T.b * dx + T.d * dy;
}

struct Img {
  int cell;
  Iso T;
};

// ------------------------------------------------------------- quadrature
void gauss_legendre01(int n, std::vector<double> &x, std::vector<double> &w) {
  x.assign(n, 0);
  w.assign(n, 0);
  for (int i = 0; i < n; i++) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; it++) {
      double p0 = 1, p1 = z;
      for (int k = 2; k <= n; k++) {
        double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      double dp = n * (z * p1 - p0) / (z * z - 1);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1, p1 = z;
    for (int k = 2; k <= n; k++) {
      double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    double dp = n * (z * p1 - p0) / (z * z - 1);
    x[i] = 0.5 * (1 - z);
    w[i] = 1.0 / ((1 - z * z) * dp * dp);  // half of the [-1,1] weight
  }
}

// collapsed 4x4 Gauss rule on {a, b >= 0, a + b <= 1}: exact to total degree 6
struct TriRule {
  std::vector<double> a, b, w;
};
const TriRule &tri_rule() {
  static TriRule r = [] {
    TriRule t;
    std::vector<double> x, w;
    gauss_legendre01(4, x, w);
    double s = 0;
    for (int i = 0; i < 4; i++)
      for (int j = 0; j < 4; j++) {
        t.a.push_back(x[i]);
        t.b.push_back(x[j] * (1 - x[i]));
        t.w.push_back(w[i] * w[j] * (1 - x[i]));
        s += t.w.back();
      }
    for (auto &v : t.w) v /= s;
    return t;
  }();
  return r;
}

// ------------------------------------------------- P3 Taylor monomial basis
void mono(double x, double y, double m[10]) {
  m[0] = 1; m[1] = x; m[2] = y; m[3] = 0.5 * x * x; m[4] = x * y; m[5] = 0.5 * y * y;
  m[6] = x * x * x / 6; m[7] = 0.5 * x * x * y; m[8] = 0.5 * x * y * y; m[9] = y * y * y / 6;
}
void mono_dx(double x, double y, double m[10]) {
  m[0] = 0; m[1] = 1; m[2] = 0; m[3] = x; m[4] = y; m[5] = 0;
  m[6] = 0.5 * x * x; m[7] = x * y; m[8] = 0.5 * y * y; m[9] = 0;
}
void mono_dy(double x, double y, double m[10]) {
  m[0] = 0; m[1] = 0; m[2] = 1; m[3] = 0; m[4] = x; m[5] = y;
  m[6] = 0; m[7] = 0.5 * x * x; m[8] = x * y; m[9] = 0.5 * y * y;
}

// ---------------------------------- pseudo-inverse by Gram-Schmidt (twice)
// A (m x n, row-major, m >= n) = Q R; P = R^-1 Q^T (n x m, row-major).
bool pinv_mgs(int m, int n, const double *A, double *P) {
  std::vector<double> Q(A, A + m * n), R(n * n, 0.0);
  for (int k = 0; k < n; k++) {
    for (int pass = 0; pass < 2; pass++)
      for (int i = 0; i < k; i++) {
        double s = 0;
        for (int r = 0; r < m; r++) s += Q[r * n + i] * Q[r * n + k];
        for (int r = 0; r < m; r++) Q[r * n + k] -= s * Q[r * n + i];
        R[i * n + k] += s;
      }
    double nr = 0;
    for (int r = 0; r < m; r++) nr += Q[r * n + k] * Q[r * n + k];
    nr = std::sqrt(nr);
    if (!(nr > 0)) return false;
    R[k * n + k] = nr;
    for (int r = 0; r < m; r++) Q[r * n + k] /= nr;
  }
  // P = R^-1 Q^T by back substitution, column by column of Q^T
  for (int c = 0; c < m; c++)
    for (int i = n - 1; i >= 0; i--) {
      double s = Q[c * n + i];
      for (int j = i + 1; j < n; j++) s -= R[i * n + j] * P[j * m + c];
      P[i * m + c] = s / R[i * n + i];
    }
  return true;
}

struct Cell {
  double p[3][2];
  double cx, cy, area, hs;
  int v[3];        // global vertex ids
  int8_t bc[3];
};

void cell_xi(const Cell &c, double x, double y, double &xi, double &eta) {
  xi = (x - c.cx) / c.hs;
  eta = (y - c.cy) / c.hs;
}

// average over triangle P (viewer frame) of the monomials of cell c (and derivatives)
void tri_avg(const Cell &c, const double P[3][2], double am[10], double ax[10], double ay[10]) {
  const TriRule &r = tri_rule();
  for (int k = 0; k < 10; k++) am[k] = ax[k] = ay[k] = 0;
  for (size_t q = 0; q < r.w.size(); q++) {
    double x = P[0][0] + r.a[q] * (P[1][0] - P[0][0]) + r.b[q] * (P[2][0] - P[0][0]);
    double y = P[0][1] + r.a[q] * (P[1][1] - P[0][1]) + r.b[q] * (P[2][1] - P[0][1]);
    double xi, eta, m[10], mx[10], my[10];
    cell_xi(c, x, y, xi, eta);
    mono(xi, eta, m);
    mono_dx(xi, eta, mx);
    mono_dy(xi, eta, my);
    for (int k = 0; k < 10; k++) {
      am[k] += r.w[q] * m[k];
      ax[k] += r.w[q] * mx[k];
      ay[k] += r.w[q] * my[k];
    }
  }
}

void image_tri(const std::vector<Cell> &cells, const Img &im, double P[3][2]) {
  const Cell &c = cells[im.cell];
  for (int k = 0; k < 3; k++) iso_apply(im.T, c.p[k][0], c.p[k][1], P[k][0], P[k][1]);
}
void image_centroid(const std::vector<Cell> &cells, const Img &im, double &x, double &y) {
  iso_apply(im.T, cells[im.cell].cx, cells[im.cell].cy, x, y);
}

uint64_t spread_bits(uint32_t v) {
  uint64_t x = v;
  x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
  x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
  x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
  x = (x | (x << 2)) & 0x3333333333333333ull;
  x = (x | (x << 1)) & 0x5555555555555555ull;
  return x;
}

struct Face {
  int nb = -1;     // neighbour cell (device index), the cell itself for walls
  int nbk = -1;    // neighbour's local edge
  Iso T = iso_id();  // maps the neighbour's frame into this cell's frame
  int edge = -1;
  bool is_left = false;
};

}  // namespace

int prepare(int n, const gks2l_mesh *meshes, Prep &out, std::string &err) {
  Prep P;
  P.ninst = n;
  std::vector<Cell> cells;
  std::vector<int8_t> dummy;
  int vbase = 0;
  // ---- cells, per instance in Morton order
  for (int i = 0; i < n; i++) {
    const gks2l_mesh &M = meshes[i];
    if (M.n_vert <= 0 || M.n_tri <= 0 || !M.xy || !M.tri) { err = "empty mesh"; return GKS2L_EINVAL; }
    P.vert_offset.push_back(vbase);
    for (int v = 0; v < M.n_vert; v++) {
      P.vx.push_back(M.xy[2 * v]);
      P.vy.push_back(M.xy[2 * v + 1]);
    }
    std::vector<Cell> loc(M.n_tri);
    double bx0 = 1e300, by0 = 1e300, bx1 = -1e300, by1 = -1e300;
    for (int t = 0; t < M.n_tri; t++) {
      Cell &c = loc[t];
      for (int k = 0; k < 3; k++) {
        int v = M.tri[3 * t + k];
        if (v < 0 || v >= M.n_vert) { err = "vertex index out of range"; return GKS2L_EMESH; }
        c.v[k] = vbase + v;
        c.p[k][0] = M.xy[2 * v];
        c.p[k][1] = M.xy[2 * v + 1];
        c.bc[k] = M.tri_bc ? M.tri_bc[3 * t + k] : (int8_t)GKS2L_BC_INTERIOR;
      }
      double a = 0.5 * ((c.p[1][0] - c.p[0][0]) * (c.p[2][1] - c.p[0][1]) -
                        (c.p[1][1] - c.p[0][1]) * (c.p[2][0] - c.p[0][0]));
      if (!(a > 0)) { err = "triangle " + std::to_string(t) + " is not counter-clockwise"; return GKS2L_EMESH; }
      c.area = a;
      c.hs = std::sqrt(a);
      c.cx = (c.p[0][0] + c.p[1][0] + c.p[2][0]) / 3;
      c.cy = (c.p[0][1] + c.p[1][1] + c.p[2][1]) / 3;
      bx0 = std::min(bx0, c.cx); bx1 = std::max(bx1, c.cx);
      by0 = std::min(by0, c.cy); by1 = std::max(by1, c.cy);
    }
    double sx = bx1 > bx0 ? (bx1 - bx0) : 1, sy = by1 > by0 ? (by1 - by0) : 1;
    std::vector<uint64_t> key(M.n_tri);
    for (int t = 0; t < M.n_tri; t++) {
      uint32_t qx = (uint32_t)std::min(4294967295.0, std::floor((loc[t].cx - bx0) / sx * 4294967295.0));
      uint32_t qy = (uint32_t)std::min(4294967295.0, std::floor((loc[t].cy - by0) / sy * 4294967295.0));
      // Morton key of the top 16 bits of each quantised centroid coordinate
      key[t] = spread_bits(qx >> 16) | (spread_bits(qy >> 16) << 1);
    }
    std::vector<int> order(M.n_tri);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return key[a] < key[b]; });
    int cbase = (int)cells.size();
    int callerbase = 0;
    for (int k = 0; k < i; k++) callerbase += meshes[k].n_tri;
    P.inst_first.push_back(cbase);
    for (int r = 0; r < M.n_tri; r++) {
      cells.push_back(loc[order[r]]);
      P.perm.push_back(callerbase + order[r]);
      P.inst.push_back(i);
    }
    vbase += M.n_vert;
  }
  P.inst_first.push_back((int)cells.size());
  P.nt = (int)cells.size();
  P.nv = vbase;
  const int nt = P.nt;

  // ---- faces: interior pairs by vertex pairs; boundary by kind
  std::vector<Face> face(3 * nt);
  {
    std::unordered_map<uint64_t, int> open;  // vertex pair -> half-edge (cell*3+k)
    open.reserve(3 * nt);
    for (int c = 0; c < nt; c++)
      for (int k = 0; k < 3; k++) {
        uint32_t a = cells[c].v[k], b = cells[c].v[(k + 1) % 3];
        uint64_t key = ((uint64_t)std::min(a, b) << 32) | std::max(a, b);
        auto it = open.find(key);
        if (it == open.end()) {
          open.emplace(key, 3 * c + k);
        } else {
          int h = it->second;
          int c2 = h / 3, k2 = h % 3;
          face[3 * c + k].nb = c2; face[3 * c + k].nbk = k2;
          face[3 * c2 + k2].nb = c; face[3 * c2 + k2].nbk = k;
          open.erase(it);
        }
      }
    // boundary half-edges left in `open`
    std::vector<int> per;
    for (auto &kv : open) {
      int h = kv.second, c = h / 3, k = h % 3;
      int kind = cells[c].bc[k];
      if (kind == GKS2L_BC_PERIODIC) {
        per.push_back(h);
      } else {
        double ax = cells[c].p[k][0], ay = cells[c].p[k][1];
        double bx = cells[c].p[(k + 1) % 3][0], by = cells[c].p[(k + 1) % 3][1];
        double l = std::hypot(bx - ax, by - ay);
        face[h].nb = c; face[h].nbk = k;
        face[h].T = iso_mirror(ax, ay, (by - ay) / l, -(bx - ax) / l);
      }
    }
    // periodic: match wrapped midpoints within each instance
    struct PE { int h, inst; double wx, wy, mx, my; };
    std::vector<PE> pes;
    for (int h : per) {
      int c = h / 3, k = h % 3, ii = P.inst[c];
      const gks2l_mesh &M = meshes[ii];
      double mx = 0.5 * (cells[c].p[k][0] + cells[c].p[(k + 1) % 3][0]);
      double my = 0.5 * (cells[c].p[k][1] + cells[c].p[(k + 1) % 3][1]);
      double x0 = 1e300, y0 = 1e300;
      for (int v = 0; v < M.n_vert; v++) { x0 = std::min(x0, M.xy[2 * v]); y0 = std::min(y0, M.xy[2 * v + 1]); }
      double wx = mx, wy = my;
      if (M.period[0] > 0) wx = mx - M.period[0] * std::floor((mx - x0) / M.period[0] + 1e-9);
      if (M.period[1] > 0) wy = my - M.period[1] * std::floor((my - y0) / M.period[1] + 1e-9);
      pes.push_back({h, ii, wx, wy, mx, my});
    }
    std::sort(pes.begin(), pes.end(), [](const PE &a, const PE &b) {
      if (a.inst != b.inst) return a.inst < b.inst;
      return a.wx < b.wx || (a.wx == b.wx && a.wy < b.wy);
    });
    std::vector<char> done(pes.size(), 0);
    for (size_t i = 0; i < pes.size(); i++) {
      if (done[i]) continue;
      const PE &p = pes[i];
      double tol = 1e-7 * cells[p.h / 3].hs;
      size_t found = pes.size();
      for (size_t j = i + 1; j < pes.size() && pes[j].inst == p.inst && pes[j].wx <= p.wx + tol; j++)
        if (!done[j] && std::fabs(pes[j].wy - p.wy) <= tol) { found = j; break; }
      if (found == pes.size()) { err = "unmatched periodic edge"; return GKS2L_EMESH; }
      done[i] = done[found] = 1;
      const PE &q = pes[found];
      int c1 = p.h / 3, k1 = p.h % 3, c2 = q.h / 3, k2 = q.h % 3;
      double sx = p.mx - q.mx, sy = p.my - q.my;  // maps c2's frame into c1's
      // the partner must be the same edge translated (end points swapped:
      // both triangles are counter-clockwise, on opposite sides)
      const double *a0 = cells[c1].p[k1], *a1 = cells[c1].p[(k1 + 1) % 3];
      const double *b0 = cells[c2].p[k2], *b1 = cells[c2].p[(k2 + 1) % 3];
      if (std::fabs(b0[0] + sx - a1[0]) > tol || std::fabs(b0[1] + sy - a1[1]) > tol ||
          std::fabs(b1[0] + sx - a0[0]) > tol || std::fabs(b1[1] + sy - a0[1]) > tol) {
        err = "periodic sides do not match";
        return GKS2L_EMESH;
      }
      face[p.h].nb = c2; face[p.h].nbk = k2; face[p.h].T = iso_shift(sx, sy);
      face[q.h].nb = c1; face[q.h].nbk = k1; face[q.h].T = iso_shift(-sx, -sy);
    }
  }
  for (int h = 0; h < 3 * nt; h++)
    if (face[h].nb < 0) { err = "face without neighbour"; return GKS2L_EMESH; }

  // ---- transform codes (linear parts)
  auto xf_code = [&](const Iso &T) -> int {
    for (int c = 0; c < P.nxf; c++) {
      const double *m = &P.xf[4 * c];
      if (std::fabs(m[0] - T.a) < 1e-12 && std::fabs(m[1] - T.b) < 1e-12 && std::fabs(m[2] - T.c) < 1e-12 &&
          std::fabs(m[3] - T.d) < 1e-12)
        return c;
    }
    if (P.nxf >= kMaxXf) return -1;
    P.xf.insert(P.xf.end(), {T.a, T.b, T.c, T.d});
    return P.nxf++;
  };
  xf_code(iso_id());

  // ---- edges in device-cell order (L = the lower index; walls: L = the cell)
  for (int c = 0; c < nt; c++)
    for (int k = 0; k < 3; k++) {
      Face &f = face[3 * c + k];
      bool wall = (f.nb == c && f.nbk == k);
      if (f.edge >= 0) continue;
      if (!wall && f.nb < c) continue;  // created from the other side
      int e = P.ne++;
      f.edge = e;
      f.is_left = true;
      if (!wall) {
        Face &g = face[3 * f.nb + f.nbk];
        g.edge = e;
        g.is_left = false;
      }
      const Cell &L = cells[c];
      double ax = L.p[k][0], ay = L.p[k][1], bx = L.p[(k + 1) % 3][0], by = L.p[(k + 1) % 3][1];
      double dx = bx - ax, dy = by - ay, len = std::hypot(dx, dy);
      P.eL.push_back(c);
      P.eR.push_back(f.nb);
      int code = xf_code(f.T);
      if (code < 0) { err = "too many distinct image transforms"; return GKS2L_EMESH; }
      P.exf.push_back((int8_t)code);
      P.en0.push_back(dy / len);
      P.en1.push_back(-dx / len);
      P.elen.push_back(len);
      P.ev0.push_back(L.v[k]);
      P.ev1.push_back(L.v[(k + 1) % 3]);
      const double gs[2] = {0.5 - 0.5 / std::sqrt(3.0), 0.5 + 0.5 / std::sqrt(3.0)};
      for (int q = 0; q < 2; q++) {
        double x = ax + gs[q] * dx, y = ay + gs[q] * dy;
        double xi, eta, xr, yr;
        cell_xi(L, x, y, xi, eta);
        P.exiL.push_back(xi);
        P.exiL.push_back(eta);
        iso_apply_inv(f.T, x, y, xr, yr);
        cell_xi(cells[f.nb], xr, yr, xi, eta);
        P.exiR.push_back(xi);
        P.exiR.push_back(eta);
      }
    }
  const int ne = P.ne;
  // exiL/exiR were pushed edge-major with 4 values; transpose to [4][edge]
  {
    std::vector<double> a(4 * ne), b(4 * ne);
    for (int e = 0; e < ne; e++)
      for (int q = 0; q < 4; q++) { a[q * ne + e] = P.exiL[4 * e + q]; b[q * ne + e] = P.exiR[4 * e + q]; }
    P.exiL.swap(a);
    P.exiR.swap(b);
  }

  // ---- per-cell operators
  P.area.resize(nt); P.hs.resize(nt); P.dX.resize(nt);
  P.vtx.resize(3 * nt);
  P.st_cell.assign(kSlots * nt, -1);
  P.st_xf.assign(kSlots * nt, 0);
  P.lsq.assign(kCoef * kCols * nt, 0.0);
  P.p1op.assign(30 * nt, 0.0);
  P.bq.assign(kBeta * nt, 0.0);
  P.mmean.assign(7 * nt, 0.0);
  P.plane.assign(6 * nt, 0.0);
  P.cedge.assign(3 * nt, 0);
  const TriRule &rule = tri_rule();
  // first pass (serial: it registers image transforms): geometry and the
  // compact stencil of every cell
  std::vector<Img> lists((size_t)kSlots * nt);
  std::vector<int> nlist(nt);
  for (int j = 0; j < nt; j++) {
    const Cell &C = cells[j];
    P.area[j] = C.area;
    P.hs[j] = C.hs;
    double per = 0;
    for (int k = 0; k < 3; k++) {
      per += std::hypot(C.p[(k + 1) % 3][0] - C.p[k][0], C.p[(k + 1) % 3][1] - C.p[k][1]);
      P.vtx[3 * j + k] = C.v[k];
      const Face &f = face[3 * j + k];
      P.cedge[k * nt + j] = f.is_left ? f.edge : ~f.edge;
    }
    P.dX[j] = 4 * C.area / per;
    // compact stencil: face images then their other neighbours, deduplicated
    Img list[kSlots];
    int na = 0;
    double tol = 1e-8 * C.hs;
    auto same = [&](const Img &a, double x, double y) {
      double ax, ay;
      image_centroid(cells, a, ax, ay);
      return std::fabs(ax - x) <= tol && std::fabs(ay - y) <= tol;
    };
    for (int k = 0; k < 3; k++) list[na++] = {face[3 * j + k].nb, face[3 * j + k].T};
    for (int k = 0; k < 3; k++) {
      Img fi = list[k];
      for (int g = 0; g < 3; g++) {
        const Face &ff = face[3 * fi.cell + g];
        Img cand{ff.nb, iso_mul(fi.T, ff.T)};
        double cx, cy;
        image_centroid(cells, cand, cx, cy);
        if (cand.cell == j && std::fabs(cx - C.cx) <= tol && std::fabs(cy - C.cy) <= tol) continue;
        bool dup = false;
        for (int s = 0; s < na; s++)
          if (list[s].cell == cand.cell && same(list[s], cx, cy)) { dup = true; break; }
        if (dup) continue;
        if (na >= kSlots) { err = "stencil overflow"; return GKS2L_EMESH; }
        list[na++] = cand;
      }
    }
    for (int s = 0; s < na; s++) {
      P.st_cell[s * nt + j] = list[s].cell;
      int code = xf_code(list[s].T);
      if (code < 0) { err = "too many distinct image transforms"; return GKS2L_EMESH; }
      P.st_xf[s * nt + j] = (int8_t)code;
      lists[(size_t)kSlots * j + s] = list[s];
    }
    nlist[j] = na;
  }
  // second pass (threads over cell ranges): the per-cell operators
  auto ops = [&](int j0, int j1, std::string &terr) {
  for (int j = j0; j < j1; j++) {
    const Cell &C = cells[j];
    const Img *list = &lists[(size_t)kSlots * j];
    const int na = nlist[j];
    // LS system: averages of the zero-mean basis over the stencil images,
    // then h-scaled average derivatives over the cell and its faces
    double am[10], ax[10], ay[10];
    tri_avg(C, C.p, am, ax, ay);
    for (int k = 3; k < 10; k++) P.mmean[(k - 3) * nt + j] = am[k];
    int m = na + 8;
    std::vector<double> A(m * kCoef), Pm(kCoef * m);
    for (int s = 0; s < na; s++) {
      double T[3][2], im[10], ix[10], iy[10];
      image_tri(cells, list[s], T);
      tri_avg(C, T, im, ix, iy);
      for (int k = 1; k < 10; k++) A[s * kCoef + k - 1] = im[k] - am[k];
    }
    for (int f = 0; f < 4; f++) {
      double T[3][2], im[10], ix[10], iy[10];
      if (f == 0) std::memcpy(T, C.p, sizeof(T));
      else image_tri(cells, list[f - 1], T);
      tri_avg(C, T, im, ix, iy);
      for (int k = 1; k < 10; k++) {
        A[(na + 2 * f) * kCoef + k - 1] = ix[k];
        A[(na + 2 * f + 1) * kCoef + k - 1] = iy[k];
      }
    }
    if (!pinv_mgs(m, kCoef, A.data(), Pm.data())) { terr = "singular least-squares system"; return; }
    for (int r = 0; r < kCoef; r++) {
      for (int s = 0; s < na; s++) P.lsq[(r * kCols + s) * nt + j] = Pm[r * m + s];
      for (int c = 0; c < 8; c++) P.lsq[(r * kCols + 9 + c) * nt + j] = Pm[r * m + na + c];
    }
    // P1 sub-stencils {cell, face f}
    for (int f = 0; f < 3; f++) {
      double T[3][2], im[10], ix[10], iy[10];
      image_tri(cells, list[f], T);
      tri_avg(C, T, im, ix, iy);
      double B5[10] = {im[1] - am[1], im[2] - am[2], 1, 0, 0, 1, 1, 0, 0, 1}, P5[10];
      if (!pinv_mgs(5, 2, B5, P5)) { terr = "singular P1 system"; return; }
      for (int q = 0; q < 10; q++) P.p1op[(f * 10 + q) * nt + j] = P5[q];
    }
    // smoothness form: mean over the cell of squared xi-derivatives of
    // orders 1 and 2, plus the (constant) third derivatives
    double Bq[9][9] = {{0}};
    for (size_t q = 0; q < rule.w.size(); q++) {
      double x = C.p[0][0] + rule.a[q] * (C.p[1][0] - C.p[0][0]) + rule.b[q] * (C.p[2][0] - C.p[0][0]);
      double y = C.p[0][1] + rule.a[q] * (C.p[1][1] - C.p[0][1]) + rule.b[q] * (C.p[2][1] - C.p[0][1]);
      double X, Y;
      cell_xi(C, x, y, X, Y);
      double d[5][9] = {
          {1, 0, X, Y, 0, 0.5 * X * X, X * Y, 0.5 * Y * Y, 0},   // d/dxi
          {0, 1, 0, X, Y, 0, 0.5 * X * X, X * Y, 0.5 * Y * Y},   // d/deta
          {0, 0, 1, 0, 0, X, Y, 0, 0},                           // d2/dxi2
          {0, 0, 0, 1, 0, 0, X, Y, 0},                           // d2/dxi deta
          {0, 0, 0, 0, 1, 0, 0, X, Y}};                          // d2/deta2
      for (int a = 0; a < 9; a++)
        for (int b = 0; b < 9; b++) {
          double s = 0;
          for (int r = 0; r < 5; r++) s += d[r][a] * d[r][b];
          Bq[a][b] += rule.w[q] * s;
        }
    }
    for (int a = 5; a < 9; a++) Bq[a][a] += 1.0;
    int idx = 0;
    for (int a = 0; a < 9; a++)
      for (int b = a; b < 9; b++) P.bq[(idx++) * nt + j] = (a == b ? 1.0 : 2.0) * Bq[a][b];
    // plane through the three edge centres: gradient = sum_f c_f v_f
    double mxy[3][2];
    for (int f = 0; f < 3; f++) {
      mxy[f][0] = 0.5 * (C.p[f][0] + C.p[(f + 1) % 3][0]);
      mxy[f][1] = 0.5 * (C.p[f][1] + C.p[(f + 1) % 3][1]);
    }
    double a11 = mxy[1][0] - mxy[0][0], a12 = mxy[1][1] - mxy[0][1];
    double a21 = mxy[2][0] - mxy[0][0], a22 = mxy[2][1] - mxy[0][1];
    double det = a11 * a22 - a12 * a21;
    // g = A^-1 [v1 - v0; v2 - v0], A rows (a11 a12), (a21 a22)
    double i11 = a22 / det, i12 = -a12 / det, i21 = -a21 / det, i22 = a11 / det;
    double c1[2] = {i11, i21}, c2[2] = {i12, i22};
    for (int d = 0; d < 2; d++) {
      P.plane[(0 * 2 + d) * nt + j] = -c1[d] - c2[d];
      P.plane[(1 * 2 + d) * nt + j] = c1[d];
      P.plane[(2 * 2 + d) * nt + j] = c2[d];
    }
  }
  };
  const int nth = (int)std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  const int chunk = (nt + nth - 1) / nth;
  std::vector<std::string> terrs(nth);
  std::vector<std::thread> pool;
  for (int t = 0; t < nth && t * chunk < nt; t++)
    pool.emplace_back(ops, t * chunk, std::min(nt, (t + 1) * chunk), std::ref(terrs[t]));
  for (auto &th : pool) th.join();
  for (auto &e : terrs)
    if (!e.empty()) { err = e; return GKS2L_EMESH; }
  out = std::move(P);
  return GKS2L_OK;
}

void bathymetry(const Prep &p, const double *bvert, std::vector<double> &bmean, std::vector<double> &bgx,
                std::vector<double> &bgy, std::vector<double> &eb0, std::vector<double> &eb1) {
  const int nt = p.nt, ne = p.ne;
  bmean.resize(nt); bgx.resize(nt); bgy.resize(nt);
  for (int j = 0; j < nt; j++) {
    int v0 = p.vtx[3 * j], v1 = p.vtx[3 * j + 1], v2 = p.vtx[3 * j + 2];
    double b0 = bvert ? bvert[v0] : 0, b1 = bvert ? bvert[v1] : 0, b2 = bvert ? bvert[v2] : 0;
    bmean[j] = (b0 + b1 + b2) / 3;
    double d1x = p.vx[v1] - p.vx[v0], d1y = p.vy[v1] - p.vy[v0];
    double d2x = p.vx[v2] - p.vx[v0], d2y = p.vy[v2] - p.vy[v0];
    double det = d1x * d2y - d1y * d2x;
    double f1 = b1 - b0, f2 = b2 - b0;
    bgx[j] = (f1 * d2y - f2 * d1y) / det;
    bgy[j] = (f2 * d1x - f1 * d2x) / det;
  }
  eb0.resize(ne); eb1.resize(ne);
  const double gs[2] = {0.5 - 0.5 / std::sqrt(3.0), 0.5 + 0.5 / std::sqrt(3.0)};
  for (int e = 0; e < ne; e++) {
    double ba = bvert ? bvert[p.ev0[e]] : 0, bb = bvert ? bvert[p.ev1[e]] : 0;
    eb0[e] = ba + gs[0] * (bb - ba);
    eb1[e] = ba + gs[1] * (bb - ba);
  }
}

}  // namespace gks2l
