// Host-side mesh preparation for the gks2l device path: renumbering, edges,
// compact stencils, least-squares operators and per-edge geometry, laid out as
// structure-of-arrays in the device order. Internal header of the library.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "gks2l.h"

namespace gks2l {

constexpr int kSlots = 9;        // average rows of the P3 system (cells i, j, k + neighbours)
constexpr int kCols = 17;        // 9 average columns + 8 gradient columns
constexpr int kCoef = 9;         // P3 unknowns a_1..a_9 (a_0 = cell average)
constexpr int kBeta = 45;        // upper triangle of the 9x9 smoothness form
constexpr int kMaxXf = 64;       // distinct linear parts of image transforms

struct Prep {
  int nt = 0, ne = 0, nv = 0, ninst = 0;
  std::vector<int> perm;         // device cell -> caller cell
  std::vector<int> inst;         // instance of each device cell
  std::vector<int> inst_first;   // first device cell of each instance (+ end)
  std::vector<int> vtx;          // 3 per cell: global vertex ids (device order)
  std::vector<int> vert_offset;  // first global vertex of each instance
  std::vector<double> vx, vy;    // global vertex coordinates
  // per cell
  std::vector<double> area, hs, dX;
  std::vector<int> st_cell;      // [slot][cell]
  std::vector<int8_t> st_xf;     // [slot][cell]
  std::vector<double> lsq;       // [row*17+col][cell]
  std::vector<double> p1op;      // [(f*2+d)*5+c][cell]
  std::vector<double> bq;        // [45][cell]
  std::vector<double> mmean;     // [7][cell] means of monomials 3..9
  std::vector<double> plane;     // [(f*2+d)][cell]
  std::vector<int> cedge;        // [f][cell]: edge id, or ~edge when the cell is the edge's R side
  // per edge
  std::vector<int> eL, eR;
  std::vector<int8_t> exf;       // transform of the R side (0 = identity)
  std::vector<double> en0, en1, elen;
  std::vector<double> exiL, exiR;  // [4][edge]: Gauss points in each side's scaled frame
  std::vector<int> ev0, ev1;     // edge end vertices (global), for B along the edge
  std::vector<double> xf;        // [code*4]: 2x2 linear parts of the image transforms
  int nxf = 0;
};

// Build the preparation for n meshes (an ensemble is a disjoint union).
// Returns GKS2L_OK or GKS2L_EMESH with a message in err.
int prepare(int n, const gks2l_mesh *meshes, Prep &out, std::string &err);

// Bathymetry derived data from vertex samples (global vertex order):
// per cell mean and P1 gradient, per edge the two Gauss-point values.
void bathymetry(const Prep &p, const double *bvert,
                std::vector<double> &bmean, std::vector<double> &bgx, std::vector<double> &bgy,
                std::vector<double> &eb0, std::vector<double> &eb1);

}  // namespace gks2l
