// Host-side data structures of the cut-cell setup (geometry, discretisation, hierarchy).
#pragma once

#include <array>
#include <memory>
#include <cstdint>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/ccm.h"

namespace ccm {

constexpr int NMOM = 15;                        // monomials x^p y^q with p + q <= 4
using Mom = std::array<double, NMOM>;

// graded order (0,0),(1,0),(0,1),(2,0),(1,1),(0,2),(3,0),...
inline int mono_p(int k) {
  static const int P[NMOM] = {0, 1, 0, 2, 1, 0, 3, 2, 1, 0, 4, 3, 2, 1, 0};
  return P[k];
}
inline int mono_q(int k) {
  static const int Q[NMOM] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3, 0, 1, 2, 3, 4};
  return Q[k];
}
inline int mono_index(int p, int q) { int d = p + q; return d * (d + 1) / 2 + q; }

enum CellStatus : int8_t { ST_EMPTY = 0, ST_PURE = 1, ST_CUT = 2 };

struct Error {
  int code;
  std::string msg;
};

struct Curve {
  int kind = 0;
  double p[8] = {0};
  int orient = -1;
  int bc = CCM_DIRICHLET;
  double robin[2] = {1.0, 0.0};     // CCM_ROBIN: gamma1, gamma2 of gamma1 u + gamma2 du/dn
  std::vector<double> V;            // CCM_POLYGON, CCM_SPLINE: points (x, y) counter-clockwise
  std::vector<double> knots, M[2];  // CCM_SPLINE: knots t_0 = 0 .. t_n = 2 pi; second derivatives
  std::vector<double> poly;         // CCM_SPLINE: 64 samples per cubic (the inside test)
  bool prepare();                   // CCM_SPLINE: knots and second derivatives from V
  void xy(double t, double& x, double& y) const;
  void dxy(double t, double& x, double& y) const;
  bool inside(double x, double y) const;   // strictly inside the closed curve
  // [t0, t1] (either direction) cut at the curve's kinks, in the order of traversal
  void subintervals(double t0, double t1, std::vector<std::pair<double, double>>& out) const;
};

// A piece of a cut-cell boundary in global coordinates, traversed with Omega on its left.
struct Piece {
  bool arc = false;
  int curve = -1;
  double t0 = 0, t1 = 0;            // arc parameters, from t0 to t1
  double ax = 0, ay = 0, bx = 0, by = 0;  // straight segment from (ax, ay) to (bx, by)
  bool wall = false;                // straight piece on a box wall that is part of dOmega
};

struct Region {
  std::vector<Piece> pieces;
  int hi = 0, hj = 0;               // Cartesian cell the loop was built in
  Mom mom{};                        // moments in the frame of (hi, hj)
};

// Geometry of one level: cut cells after Alg. 1.
struct CutLevel {
  int nx = 0, ny = 0;
  double x0 = 0, y0 = 0, h = 0;
  int box_bc = CCM_NONE;
  std::vector<Curve> curves;
  std::vector<int8_t> status;       // [ny*nx] post-merge status
  std::vector<int32_t> owner;       // survivor linear index, -1 if empty
  std::vector<double> vol;          // volume / h^2, 0 for empty
  std::vector<uint8_t> iface;       // pre-merge interface cells
  std::unordered_map<int, std::vector<Region>> regions;   // non-pure survivors
  std::unordered_map<int, Mom> mom;                      // non-pure survivors, own frame
  std::unordered_map<int, int> first_curve;              // pre-merge interface cell -> curve
  std::unordered_map<int, double> arc_param;             // pre-merge interface cell -> mid t
  // boundary segments (sorted by cell index)
  std::vector<int> segs;
  std::unordered_map<int, int> seg_of;
  std::vector<int> seg_bc;
  std::vector<std::array<double, 2>> seg_gamma;   // the segment's operator gamma1 u + gamma2 du/dn
  std::vector<Mom> bm0, bmx, bmy;
  std::vector<std::vector<Piece>> seg_pieces;

  double cx(int i) const { return x0 + (i + 0.5) * h; }
  double cy(int j) const { return y0 + (j + 0.5) * h; }
  const Mom& moments(int lin) const;
};

// Fitted rows of one level (h^2-scaled coefficients).
struct Rows {
  std::vector<uint8_t> regular;     // [ny*nx]
  std::vector<int> irr;             // linear indices of irregular cells (row-major order)
  std::vector<std::array<int, 15>> cols;     // stencil cells (linear indices), cell i first
  std::vector<std::array<double, 15>> beta;  // h^2-scaled coefficients
  std::vector<double> nb;           // h^2-scaled boundary coefficient (0 if no segment)
  std::vector<int> seg;             // segment index or -1
  double cond_max = 0;
};

const Mom& pure_moments();
Mom shift_moments(const Mom& m, double dx, double dy);
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w);

// Classification of every cell by its centre (the O(h^-2) scan of the cut-cell setup: a cell
// the boundary does not enter is pure when its centre is inside every curve that bounds Omega
// from outside and outside every hole), for a setup that runs it off the host threads
// (fitdev.cu).  status[j * nx + i] = ST_PURE or ST_EMPTY for the level's curves, box and h.
// The interface cells, whose status the crossings decide, are overwritten afterwards, and a
// centre that two evaluations of the curve could classify differently lies on the curve, so
// inside an interface cell: the result equals the host scan's.
struct CentreClassifier {
  virtual ~CentreClassifier() = default;
  virtual int classify(const CutLevel& cg, std::vector<int8_t>& status) = 0;
};
std::unique_ptr<CentreClassifier> make_device_classifier();

// geometry.cpp
// CCM_OK, or CCM_EINVAL for a problem the method does not define (sizes, ellipticity, kinds)
int check_problem(const ccm_problem& prob);
int build_cut_level(const ccm_problem& prob, int nx, int ny, double h, double theta, CutLevel& out,
                    std::string& err, CentreClassifier* cc = nullptr);
// Fits of many (fitted row, candidate PLG stencil) pairs in one call, for a setup that runs
// them off the host threads (fitdev.cu).  Pair k fits the row of cell row_cell[k] over the 15
// cells cand[k] with the host fit's arithmetic (to rounding): beta[16 k + q], norm[k] (the
// weighted norm the stencil choice compares) and ok[k] (0: the normal equations are not
// positive definite).  cond() writes the 2-norm condition number of each pair's 15 x 15 FV
// sample matrix.  Both return CCM_OK or a CCM_* error code.
struct FitBatcher {
  virtual ~FitBatcher() = default;
  virtual int fit(const CutLevel& cg, double a, double b, double c, const std::vector<int32_t>& row_cell,
                  const std::vector<std::array<int, 15>>& cand, std::vector<double>& beta, std::vector<double>& norm,
                  std::vector<uint8_t>& ok) = 0;
  virtual int cond(const CutLevel& cg, const std::vector<int32_t>& row_cell,
                   const std::vector<std::array<int, 15>>& cand, std::vector<double>& cond) = 0;
};

// fitdev.cu: the batched fits on the current CUDA device
std::unique_ptr<FitBatcher> make_device_fitter();

// discretize.cpp
// Rows of a level (Sec. 3.2 regular stencil, Sec. 3.3 fitted rows).  With fb, the candidate
// stencils are enumerated on host threads and their fits run through fb; the choice rule is
// the same.
int discretize_level(const CutLevel& cg, double a, double b, double c, int nthreads, Rows& rows,
                     std::string& err, FitBatcher* fb = nullptr);
void regular_stencil(double a, double b, double c, double w[5][5]);
// quadrature helpers for callers (geometry.cpp)
void cell_quadrature(const CutLevel& cg, std::vector<int32_t>& cell, std::vector<double>& xy,
                     std::vector<double>& w);
void boundary_quadrature(const CutLevel& cg, std::vector<int32_t>& seg, std::vector<double>& xy,
                         std::vector<double>& w, std::vector<double>& n);
// cell averages of f over every non-empty cell into out[ny * nx] (0 elsewhere): the 5 x 5
// tensor Gauss rule on pure cells, cell_quadrature on cut and merged cells; f evaluated by the
// caller in batches
void cell_averages(const CutLevel& cg, void (*f)(void*, int64_t, const double*, const double*, double*), void* ctx,
                   double* out);
// averages of gamma1 u + gamma2 du/dn over every boundary segment into out[n_segments], from
// the caller's u and gradient at the nodes of boundary_quadrature
void boundary_averages(const CutLevel& cg,
                       void (*g)(void*, int64_t, const double*, const double*, double*, double*, double*),
                       void* ctx, double* out);

}  // namespace ccm
