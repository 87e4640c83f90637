// Packed host arrays of the multigrid hierarchy (Sec. 4), ready for upload.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "host.h"

namespace ccm {

// Rows of one level ready for packing: regular mask, fitted (or transposed) rows of width W.
struct PackRows {
  int W = 15;
  std::vector<uint8_t> regular;   // [nx*ny]
  std::vector<int> irr;           // linear indices of the explicit rows' cells
  std::vector<int> cols;          // [n2*W] linear column cells (padding: the row's own cell)
  std::vector<double> beta;       // [n2*W] h^2-scaled coefficients (padding: 0)
  std::vector<double> nb;         // [n2] boundary coefficient
  std::vector<int> seg;           // [n2] boundary segment or -1
};

// Padded grid layout of one level: a 2-cell zero ring around the nx x ny cells, rows of
// `pitch` entries (a multiple of 32), cell (i, j) at (j + 2) * pitch + (i + 2).
struct HostLevel {
  int nx = 0, ny = 0, pitch = 0, rows = 0;
  double h = 0;
  long npad() const { return (long)pitch * rows; }
  long pad(int i, int j) const { return (long)(j + 2) * pitch + (i + 2); }

  std::vector<uint8_t> cls;     // [npad] 0 empty / ring, 1 regular, 2 irregular
  std::vector<double> vol;      // [npad] cell volume in units of h^2 (0 if empty)
  std::vector<int32_t> tiles;   // active 32 x 8 tiles (tile x, tile y) pairs
  std::vector<int32_t> tiles64; // active 64 x 32 tiles (TMA-staged SMO-1)

  // explicit rows, ELL with W slots: [slot][n2]
  int n2 = 0;
  int W = 15;
  std::vector<int32_t> irr_cell;   // [n2] padded index of the row's cell
  std::vector<int32_t> ell_col;    // [W * n2] padded column index
  std::vector<int32_t> ell_colf;   // the same, sign bit set for regular column cells
  std::vector<double> ell_val;     // [W * n2] h^2-scaled coefficient
  std::vector<double> nb;          // [n2] h^2-scaled boundary coefficient
  std::vector<int32_t> seg;        // [n2] boundary segment or -1

  // SMO-2 blocks: positions index `order` (row numbers of the fitted rows)
  std::vector<int32_t> order;      // [n2] rows in boundary order (Alg. 3)
  std::vector<int32_t> blk;        // [nblk * 4]: core begin, core end, ext begin, ext end
  std::vector<int64_t> blk_off;    // [nblk] offset of the block's matrix
  std::vector<double> blk_inv;     // per block [ext][core] rows of inv(L22[ext, ext]) for the core

  // coarsest level only: dense inverse over the non-empty cells
  int nb_cells = 0;
  std::vector<int32_t> bot_cell;   // [nb_cells] padded index
  std::vector<double> bot_inv;     // [nb_cells * nb_cells] stored [col][row]

  // finest level transposed rows (CSR over columns): for every padded cell that appears in a
  // fitted row, the rows referencing it
  std::vector<int32_t> tr_ptr;     // [n2col + 1]
  std::vector<int32_t> tr_cell;    // [n2col] padded index of the column cell
  std::vector<int32_t> tr_row;     // [nnz] row number
  std::vector<double> tr_val;      // [nnz] coefficient

  // user-layout maps of this level
  std::vector<int32_t> owner;      // [nx*ny] survivor linear index or -1
  std::vector<int8_t> status;      // [nx*ny]
};

struct Hierarchy {
  double a = 0, b = 0, c = 0;
  std::vector<HostLevel> levels;
  std::vector<CutLevel> cut;       // geometry of every level (kept for queries)
  std::vector<PackRows> rows;      // the rows every level was packed from
  double cond_max = 0;
  int nseg = 0;
  // wall time of the setup phases (ms): cut cells and merging, stencils and fits, the boundary
  // order with packing and the SMO-2 block inverses, the coarsest level's dense inverse
  double ms_geometry = 0, ms_fits = 0, ms_blocks = 0, ms_bottom = 0;
};

int build_hierarchy(const ccm_problem& prob, const ccm_params& par, Hierarchy& H, std::string& err,
                    FitBatcher* fb = nullptr, CentreClassifier* cc = nullptr);
// fitted rows of a level in physical units and unpadded cell indices (the layout of
// ccm_host_rows / ccm_level_rows)
int hierarchy_rows(const Hierarchy& H, int level, int32_t* cell, int32_t* cols, double* beta, double* nb,
                   int32_t* seg);
// the hierarchy of the transposed operators (L^(m))^T, on the same geometry
int build_transposed(const Hierarchy& H, const ccm_params& par, Hierarchy& T, std::string& err);
bool dense_inverse(std::vector<double>& A, int n);   // in place, partial pivoting
// SMO-2 blocks of a level's fitted rows in L.order: cores of `block` consecutive rows widened
// by `overlap` rows on each side, and the core rows of every widened block's L22 inverse
int build_smo2_blocks(HostLevel& L, int block, int overlap, int nthreads, std::string& err);

}  // namespace ccm
