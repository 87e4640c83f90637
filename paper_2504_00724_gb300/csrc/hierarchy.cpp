// Level hierarchy (Sec. 4): every level h 2^m re-embedded and re-discretised, packed for
// the device.  The irregular unknowns of each level are put in the boundary order of
// Alg. 3; SMO-2 uses overlapping blocks of that order with precomputed dense inverses of the
// L22 sub-blocks, and the coarsest level a dense inverse of L^(M).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <map>
#include <thread>
#include <atomic>

#include "hierarchy.h"

namespace ccm {

bool dense_inverse(std::vector<double>& A, int n) {
  std::vector<int> piv(n);
  std::vector<double> LU = A;
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = std::fabs(LU[(long)k * n + k]);
    for (int r = k + 1; r < n; ++r)
      if (std::fabs(LU[(long)r * n + k]) > best) {
        best = std::fabs(LU[(long)r * n + k]);
        p = r;
      }
    if (!(best > 0.0)) return false;
    piv[k] = p;
    if (p != k)
      for (int c = 0; c < n; ++c) std::swap(LU[(long)k * n + c], LU[(long)p * n + c]);
    double d = LU[(long)k * n + k];
    for (int r = k + 1; r < n; ++r) {
      double f = LU[(long)r * n + k] / d;
      LU[(long)r * n + k] = f;
      if (f != 0.0)
        for (int c = k + 1; c < n; ++c) LU[(long)r * n + c] -= f * LU[(long)k * n + c];
    }
  }
  // solve for the columns of the identity (independent: large matrices split them over threads)
  auto solve_cols = [&](int c0, int c1) {
    std::vector<double> x(n);
    for (int col = c0; col < c1; ++col) {
      std::fill(x.begin(), x.end(), 0.0);
      x[col] = 1.0;
      for (int k = 0; k < n; ++k)
        if (piv[k] != k) std::swap(x[k], x[piv[k]]);
      for (int r = 0; r < n; ++r) {
        double s = x[r];
        for (int c = 0; c < r; ++c) s -= LU[(long)r * n + c] * x[c];
        x[r] = s;
      }
      for (int r = n - 1; r >= 0; --r) {
        double s = x[r];
        for (int c = r + 1; c < n; ++c) s -= LU[(long)r * n + c] * x[c];
        x[r] = s / LU[(long)r * n + r];
      }
      for (int r = 0; r < n; ++r) A[(long)r * n + col] = x[r];
    }
  };
  const int nt = n >= 256 ? std::max(1, std::min<int>(64, (int)std::thread::hardware_concurrency())) : 1;
  if (nt == 1) {
    solve_cols(0, n);
  } else {
    std::vector<std::thread> pool;
    for (int t = 0; t < nt; ++t) pool.emplace_back(solve_cols, (int)((long)n * t / nt), (int)((long)n * (t + 1) / nt));
    for (auto& th : pool) th.join();
  }
  return true;
}

// Alg. 3: interface cells sorted by the parameter of their boundary piece (components in the
// order box, curve 0, curve 1, ...); each numbers the unnumbered irregular cells within
// Chebyshev distance 2; irregular cells farther away ride with their nearest interface cell.
static std::vector<int> boundary_order(const CutLevel& cg, const PackRows& rows) {
  const int nx = cg.nx, ny = cg.ny;
  struct Key {
    int comp;
    double s;
    int lin;
  };
  std::vector<Key> keys;
  const double W = nx * cg.h, Hh = ny * cg.h;
  // the interface cells and the pure cells with a boundary piece (box walls); the sort below
  // is a total order, so the order of collection does not matter
  for (const auto& kv : cg.first_curve) {
    const int q = kv.first;
    if (cg.iface[q]) keys.push_back({1 + kv.second, cg.arc_param.at(q), q});
  }
  for (const auto& kv : cg.seg_of) {
    const int q = kv.first;
    if (cg.iface[q] || cg.status[q] != ST_PURE) continue;
    const int j = q / nx, i = q % nx;
    double xc = cg.cx(i) - cg.x0, yc = cg.cy(j) - cg.y0;
    double d[4] = {yc, W - xc, Hh - yc, xc};
    int e = (int)(std::min_element(d, d + 4) - d);
    double s[4] = {xc, W + yc, W + Hh + (W - xc), 2 * W + Hh + (Hh - yc)};
    keys.push_back({0, s[e], q});
  }
  std::sort(keys.begin(), keys.end(), [](const Key& x, const Key& y) {
    if (x.comp != y.comp) return x.comp < y.comp;
    if (x.s != y.s) return x.s < y.s;
    return x.lin < y.lin;
  });
  std::vector<int> rowof((long)nx * ny, -1);
  for (size_t r = 0; r < rows.irr.size(); ++r) rowof[rows.irr[r]] = (int)r;
  // far cells: attach to the nearest interface cell (Chebyshev), first in key order on ties
  std::map<int, std::vector<int>> near;
  {
    std::vector<int> dist((long)nx * ny, 1 << 30), who((long)nx * ny, -1);
    // multi-source BFS in Chebyshev metric over the grid, sources in key order
    std::vector<int> frontier;
    for (size_t k = 0; k < keys.size(); ++k) {
      int q = keys[k].lin;
      if (dist[q] > 0) {
        dist[q] = 0;
        who[q] = (int)k;
        frontier.push_back(q);
      }
    }
    // only the fitted rows' cells need their nearest source: stop after the first complete
    // level of the search at which every one of them has been reached (later levels cannot
    // change the distance or the tie-break of a cell already reached)
    long unreached = 0;
    for (int q : rows.irr)
      if (dist[q] > 0) ++unreached;
    int d = 0;
    while (!frontier.empty() && unreached > 0) {
      std::vector<int> next;
      for (int q : frontier) {
        int j = q / nx, i = q % nx;
        for (int dj = -1; dj <= 1; ++dj)
          for (int di = -1; di <= 1; ++di) {
            int ii = i + di, jj = j + dj;
            if (ii < 0 || ii >= nx || jj < 0 || jj >= ny) continue;
            int q2 = jj * nx + ii;
            if (dist[q2] > d + 1) {
              if (dist[q2] == (1 << 30) && rowof[q2] >= 0) --unreached;
              dist[q2] = d + 1;
              who[q2] = who[q];
              next.push_back(q2);
            } else if (dist[q2] == d + 1 && who[q] < who[q2]) {
              who[q2] = who[q];
            }
          }
      }
      frontier.swap(next);
      ++d;
    }
    for (int q : rows.irr)
      if (dist[q] > 2 && who[q] >= 0) near[who[q]].push_back(q);
  }
  std::vector<int> order;
  std::vector<char> done(rows.irr.size(), 0);
  for (size_t k = 0; k < keys.size(); ++k) {
    int q0 = keys[k].lin, j = q0 / nx, i = q0 % nx;
    for (int dj = -2; dj <= 2; ++dj)
      for (int di = -2; di <= 2; ++di) {
        int ii = i + di, jj = j + dj;
        if (ii < 0 || ii >= nx || jj < 0 || jj >= ny) continue;
        int r = rowof[(long)jj * nx + ii];
        if (r >= 0 && !done[r]) {
          done[r] = 1;
          order.push_back(r);
        }
      }
    auto it = near.find((int)k);
    if (it != near.end())
      for (int q : it->second) {
        int r = rowof[q];
        if (r >= 0 && !done[r]) {
          done[r] = 1;
          order.push_back(r);
        }
      }
  }
  for (size_t r = 0; r < rows.irr.size(); ++r)
    if (!done[r]) order.push_back((int)r);
  return order;
}

static int pack_level(const CutLevel& cg, const PackRows& rows, const ccm_params& par, bool coarsest, bool finest,
                      HostLevel& L, std::string& err) {
  L.nx = cg.nx;
  L.ny = cg.ny;
  L.h = cg.h;
  L.pitch = ((cg.nx + 4 + 31) / 32) * 32;
  L.rows = cg.ny + 4;
  const long np = L.npad();
  L.cls.assign(np, 0);
  L.vol.assign(np, 0.0);
  L.owner = cg.owner;
  L.status = cg.status;
  for (int j = 0; j < cg.ny; ++j)
    for (int i = 0; i < cg.nx; ++i) {
      long q = (long)j * cg.nx + i;
      if (cg.status[q] == ST_EMPTY) continue;
      L.cls[L.pad(i, j)] = rows.regular[q] ? 1 : 2;
      L.vol[L.pad(i, j)] = cg.vol[q];
    }
  // active 32 x 8 tiles (any non-empty cell)
  const int tx = (cg.nx + 31) / 32, ty = (cg.ny + 7) / 8;
  L.tiles.clear();
  for (int b = 0; b < ty; ++b)
    for (int a = 0; a < tx; ++a) {
      bool any = false;
      for (int j = b * 8; j < std::min(cg.ny, b * 8 + 8) && !any; ++j)
        for (int i = a * 32; i < std::min(cg.nx, a * 32 + 32); ++i)
          if (cg.status[(long)j * cg.nx + i] != ST_EMPTY) {
            any = true;
            break;
          }
      if (any) {
        L.tiles.push_back(a);
        L.tiles.push_back(b);
      }
    }
  // active 64 x 32 tiles for the TMA-staged smoother
  {
    const int ax = (cg.nx + 63) / 64, ay = (cg.ny + 31) / 32;
    L.tiles64.clear();
    for (int b = 0; b < ay; ++b)
      for (int a = 0; a < ax; ++a) {
        bool any = false;
        for (int j = b * 32; j < std::min(cg.ny, b * 32 + 32) && !any; ++j)
          for (int i = a * 64; i < std::min(cg.nx, a * 64 + 64); ++i)
            if (rows.regular[(long)j * cg.nx + i]) {
              any = true;
              break;
            }
        if (any) {
          L.tiles64.push_back(a);
          L.tiles64.push_back(b);
        }
      }
  }
  // fitted rows
  const int n2 = (int)rows.irr.size();
  const int W = rows.W;
  L.n2 = n2;
  L.W = W;
  L.irr_cell.resize(n2);
  L.ell_col.resize((long)W * n2);
  L.ell_val.resize((long)W * n2);
  L.nb.resize(n2);
  L.seg.resize(n2);
  for (int r = 0; r < n2; ++r) {
    int q = rows.irr[r];
    L.irr_cell[r] = (int32_t)L.pad(q % cg.nx, q / cg.nx);
    for (int k = 0; k < W; ++k) {
      int c = rows.cols[(long)r * W + k];
      L.ell_col[(long)k * n2 + r] = (int32_t)L.pad(c % cg.nx, c / cg.nx);
      L.ell_val[(long)k * n2 + r] = rows.beta[(long)r * W + k];
    }
    L.nb[r] = rows.nb[r];
    L.seg[r] = rows.seg[r];
  }
  // the same columns with the sign bit set where the column cell is regular (SMO-2 reads
  // those from the new iterate and the irregular ones from the old)
  L.ell_colf.resize((long)W * n2);
  for (int r = 0; r < n2; ++r)
    for (int k = 0; k < W; ++k) {
      int c2 = rows.cols[(long)r * W + k];
      uint32_t v = (uint32_t)L.ell_col[(long)k * n2 + r];
      if (rows.regular[c2]) v |= 0x80000000u;
      L.ell_colf[(long)k * n2 + r] = (int32_t)v;
    }
  if (finest) {
    // transposed fitted rows, grouped by column cell (cells ascending; within a cell its
    // entries in row order, then slot order): a stable sort of the entries by column
    std::vector<int64_t> ent((size_t)W * n2);
    for (int r = 0; r < n2; ++r)
      for (int k = 0; k < W; ++k) ent[(size_t)r * W + k] = (size_t)r * W + k;
    auto col_of = [&](int64_t e) { return L.ell_col[(long)(e % W) * n2 + e / W]; };
    std::stable_sort(ent.begin(), ent.end(), [&](int64_t x, int64_t y) { return col_of(x) < col_of(y); });
    L.tr_ptr.assign(1, 0);
    L.tr_cell.clear();
    L.tr_row.clear();
    L.tr_val.clear();
    for (size_t i = 0; i < ent.size(); ++i) {
      const int64_t e = ent[i];
      const int r = (int)(e / W), k = (int)(e % W);
      const int32_t c = L.ell_col[(long)k * n2 + r];
      if (L.tr_cell.empty() || L.tr_cell.back() != c) {
        if (!L.tr_cell.empty()) L.tr_ptr.push_back((int32_t)L.tr_row.size());
        L.tr_cell.push_back(c);
      }
      L.tr_row.push_back(r);
      L.tr_val.push_back(L.ell_val[(long)k * n2 + r]);
    }
    if (!L.tr_cell.empty()) L.tr_ptr.push_back((int32_t)L.tr_row.size());
  }
  if (coarsest) {
    std::vector<int> cells;
    for (long q = 0; q < (long)cg.nx * cg.ny; ++q)
      if (cg.status[q] != ST_EMPTY) cells.push_back((int)q);
    const int n = (int)cells.size();
    std::vector<int> idx((long)cg.nx * cg.ny, -1);
    for (int k = 0; k < n; ++k) idx[cells[k]] = k;
    std::vector<double> A((long)n * n, 0.0);
    L.nb_cells = n;
    L.bot_cell.resize(n);
    for (int k = 0; k < n; ++k) L.bot_cell[k] = (int32_t)L.pad(cells[k] % cg.nx, cells[k] / cg.nx);
    // fill from rows: irregular rows
    std::vector<int> rowof((long)cg.nx * cg.ny, -1);
    for (int r = 0; r < n2; ++r) rowof[rows.irr[r]] = r;
    // fitted rows here; regular rows are marked and filled with the stencil by the caller
    for (int k = 0; k < n; ++k) {
      int q = cells[k];
      if (rowof[q] >= 0) {
        int r = rowof[q];
        for (int s = 0; s < W; ++s) {
          int col = idx[rows.cols[(long)r * W + s]];
          if (col < 0) {
            err = "fitted row references an empty cell";
            return CCM_EGEOM;
          }
          A[(long)k * n + col] += rows.beta[(long)r * W + s];
        }
      } else {
        A[(long)k * n + k] = NAN;
      }
    }
    L.bot_inv = A;   // finished in build_hierarchy (needs a, b, c)
  }
  // SMO-2 blocks over the boundary order
  if (!coarsest && n2 > 0) {
    // the rows were renumbered into the boundary order: blocks are contiguous row ranges
    L.order.resize(n2);
    for (int p = 0; p < n2; ++p) L.order[p] = p;
    const bool exact = n2 <= par.ras_exact;
    return build_smo2_blocks(L, exact ? n2 : par.ras_block, exact ? 0 : par.ras_overlap, par.nthreads, err);
  }
  return CCM_OK;
}

int build_smo2_blocks(HostLevel& L, int block, int overlap, int nthreads, std::string& err) {
  const int n2 = L.n2, W = L.W;
  const long np = L.npad();
  const std::vector<int32_t>& order = L.order;
  std::vector<int> pos(n2);
  for (int p = 0; p < n2; ++p) pos[order[p]] = p;
  const int m = std::max(std::min(8, n2), block), dl = std::max(0, overlap);
  const int nblk = (n2 + m - 1) / m;
  L.blk.assign(4L * nblk, 0);
  L.blk_off.assign(nblk, 0);
  long off = 0;
  for (int bk = 0; bk < nblk; ++bk) {
    int cs = bk * m, ce = std::min(n2, cs + m);
    int es = std::max(0, cs - dl), ee = std::min(n2, ce + dl);
    L.blk[4 * bk + 0] = cs;
    L.blk[4 * bk + 1] = ce;
    L.blk[4 * bk + 2] = es;
    L.blk[4 * bk + 3] = ee;
    L.blk_off[bk] = off;
    off += (long)(ee - es) * (ce - cs);
  }
  L.blk_inv.assign(off, 0.0);
  // the padded cell of every row, to look up the L22 entries
  std::vector<int> row_of_pad(np, -1);
  for (int r = 0; r < n2; ++r) row_of_pad[L.irr_cell[r]] = r;
  std::atomic<int> bad{0};
  std::atomic<int> next{0};
  int nt = nthreads > 0 ? nthreads : (int)std::max(1u, std::thread::hardware_concurrency());
  auto worker = [&]() {
    std::vector<double> A;
    while (true) {
      int bk = next.fetch_add(1);
      if (bk >= nblk) break;
      int cs = L.blk[4 * bk], ce = L.blk[4 * bk + 1], es = L.blk[4 * bk + 2], ee = L.blk[4 * bk + 3];
      int ne = ee - es;
      A.assign((long)ne * ne, 0.0);
      for (int a = 0; a < ne; ++a) {
        int r = order[es + a];
        for (int k = 0; k < W; ++k) {
          int rc = row_of_pad[L.ell_col[(long)k * n2 + r]];
          if (rc < 0) continue;                 // a regular column: L21
          int pc = pos[rc] - es;
          if (pc < 0 || pc >= ne) continue;     // outside the block
          A[(long)a * ne + pc] += L.ell_val[(long)k * n2 + r];
        }
      }
      if (!dense_inverse(A, ne)) {
        bad.store(1);
        continue;
      }
      double* dst = &L.blk_inv[L.blk_off[bk]];
      int nc = ce - cs;
      for (int e = 0; e < ne; ++e)
        for (int c = 0; c < nc; ++c) dst[(long)e * nc + c] = A[(long)(cs - es + c) * ne + e];
    }
  };
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t) th.emplace_back(worker);
  for (auto& t : th) t.join();
  if (bad.load()) {
    err = "singular L22 block";
    return CCM_ESINGULAR;
  }
  return CCM_OK;
}

// Coarsest level: fill the regular rows of the dense operator with the stencil (the packing
// marked them with NaN on the diagonal), invert, store [col][row] for coalesced reads.
static int finish_bottom(HostLevel& L, const CutLevel& cg, const double w[5][5], std::string& err) {
  const int n = L.nb_cells;
  std::vector<int> idx((long)cg.nx * cg.ny, -1);
  std::vector<int> cells;
  for (long q = 0; q < (long)cg.nx * cg.ny; ++q)
    if (cg.status[q] != ST_EMPTY) {
      idx[q] = (int)cells.size();
      cells.push_back((int)q);
    }
  std::vector<double>& A = L.bot_inv;
  for (int k = 0; k < n; ++k) {
    if (!std::isnan(A[(long)k * n + k])) continue;
    A[(long)k * n + k] = 0.0;
    int q = cells[k], j = q / cg.nx, i = q % cg.nx;
    for (int dj = -2; dj <= 2; ++dj)
      for (int di = -2; di <= 2; ++di) {
        if (w[dj + 2][di + 2] == 0.0) continue;
        int col = idx[(long)(j + dj) * cg.nx + (i + di)];
        A[(long)k * n + col] += w[dj + 2][di + 2];
      }
  }
  if (!dense_inverse(A, n)) {
    err = "singular coarsest-level operator";
    return CCM_ESINGULAR;
  }
  std::vector<double> T((long)n * n);
  for (int r = 0; r < n; ++r)
    for (int c2 = 0; c2 < n; ++c2) T[(long)c2 * n + r] = A[(long)r * n + c2];
  A.swap(T);
  return CCM_OK;
}

// Rows of the transposed operator of one level.  Column c of L collects the regular rows p
// with |p - c| <= 2 (coefficient w_{c - p}) and the fitted rows that use c.  A cell keeps the
// plain stencil in L^T (the stencil is point-symmetric) when it is regular, every cell within
// distance 2 is regular and no fitted row uses it; every other non-empty cell gets an
// explicit transposed row.
static PackRows transpose_rows(const CutLevel& cg, const PackRows& F, const double w[5][5]) {
  const int nx = cg.nx, ny = cg.ny;
  const long N = (long)nx * ny;
  const int W0 = F.W;
  std::vector<uint8_t> refd(N, 0);
  struct Ref {
    int c, p;
    double v;
  };
  std::vector<Ref> refs;
  for (size_t r = 0; r < F.irr.size(); ++r)
    for (int k = 0; k < W0; ++k) {
      const double v = F.beta[r * W0 + k];
      if (v == 0.0) continue;
      const int c = F.cols[r * W0 + k];
      refd[c] = 1;
      refs.push_back({c, F.irr[r], v});
    }
  std::sort(refs.begin(), refs.end(), [](const Ref& a, const Ref& b) { return a.c != b.c ? a.c < b.c : a.p < b.p; });
  PackRows T;
  T.regular.assign(N, 0);
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      const long q = (long)j * nx + i;
      if (!F.regular[q] || refd[q]) continue;
      bool all = true;
      for (int dj = -2; dj <= 2 && all; ++dj)
        for (int di = -2; di <= 2; ++di) {
          const int ii = i + di, jj = j + dj;
          if (ii < 0 || jj < 0 || ii >= nx || jj >= ny || !F.regular[(long)jj * nx + ii]) {
            all = false;
            break;
          }
        }
      T.regular[q] = all ? 1 : 0;
    }
  std::vector<std::vector<std::pair<int, double>>> rowsT;
  size_t rp = 0;
  int W = 1;
  for (long q = 0; q < N; ++q) {
    while (rp < refs.size() && refs[rp].c < q) ++rp;
    if (cg.status[q] == ST_EMPTY || T.regular[q]) continue;
    std::vector<std::pair<int, double>> e;
    const int j = (int)(q / nx), i = (int)(q % nx);
    for (int dj = -2; dj <= 2; ++dj)
      for (int di = -2; di <= 2; ++di) {
        const double v = w[dj + 2][di + 2];
        const int pi = i - di, pj = j - dj;
        if (v == 0.0 || pi < 0 || pj < 0 || pi >= nx || pj >= ny) continue;
        const long p = (long)pj * nx + pi;
        if (F.regular[p]) e.push_back({(int)p, v});
      }
    for (size_t k = rp; k < refs.size() && refs[k].c == q; ++k) e.push_back({refs[k].p, refs[k].v});
    W = std::max<int>(W, (int)e.size());
    T.irr.push_back((int)q);
    rowsT.push_back(std::move(e));
  }
  T.W = W;
  for (size_t r = 0; r < T.irr.size(); ++r) {
    for (int k = 0; k < W; ++k) {
      if (k < (int)rowsT[r].size()) {
        T.cols.push_back(rowsT[r][k].first);
        T.beta.push_back(rowsT[r][k].second);
      } else {
        T.cols.push_back(T.irr[r]);
        T.beta.push_back(0.0);
      }
    }
    T.nb.push_back(0.0);
    T.seg.push_back(-1);
  }
  return T;
}

int hierarchy_rows(const Hierarchy& H, int level, int32_t* cell, int32_t* cols, double* beta, double* nb,
                   int32_t* seg) {
  if (level < 0 || level >= (int)H.levels.size()) return CCM_EINVAL;
  const HostLevel& L = H.levels[level];
  const int n2 = L.n2;
  const double ih2 = 1.0 / (L.h * L.h);
  auto unpad = [&](int32_t p) { return (p / L.pitch - 2) * L.nx + (p % L.pitch - 2); };
  for (int r = 0; r < n2; ++r) {
    if (cell) cell[r] = unpad(L.irr_cell[r]);
    for (int k = 0; k < 15; ++k) {
      if (cols) cols[(long)r * 15 + k] = unpad(L.ell_col[(long)k * n2 + r]);
      if (beta) beta[(long)r * 15 + k] = L.ell_val[(long)k * n2 + r] * ih2;
    }
    if (nb) nb[r] = L.nb[r] * ih2;
    if (seg) seg[r] = L.seg[r];
  }
  return CCM_OK;
}

int build_hierarchy(const ccm_problem& prob, const ccm_params& par, Hierarchy& H, std::string& err, FitBatcher* fb,
                    CentreClassifier* cc) {
  H.a = prob.a;
  H.b = prob.b;
  H.c = prob.c;
  int nl = 1;
  while ((prob.nx >> (nl - 1)) > par.coarsest && ((prob.nx >> nl) << nl) == prob.nx && ((prob.ny >> nl) << nl) == prob.ny)
    ++nl;
  H.levels.resize(nl);
  H.cut.resize(nl);
  H.cond_max = 0;
  double w[5][5];
  regular_stencil(prob.a, prob.b, prob.c, w);
  using clk = std::chrono::steady_clock;
  auto ms_since = [](clk::time_point t) { return std::chrono::duration<double, std::milli>(clk::now() - t).count(); };
  H.ms_geometry = H.ms_fits = H.ms_blocks = H.ms_bottom = 0;
  for (int m = 0; m < nl; ++m) {
    CutLevel& cg = H.cut[m];
    auto t0 = clk::now();
    int rc = build_cut_level(prob, prob.nx >> m, prob.ny >> m, prob.h * (double)(1 << m), par.theta, cg, err, cc);
    H.ms_geometry += ms_since(t0);
    if (rc) return rc;
    Rows fit;
    t0 = clk::now();
    rc = discretize_level(cg, prob.a, prob.b, prob.c, par.nthreads, fit, err, fb);
    H.ms_fits += ms_since(t0);
    if (rc) return rc;
    t0 = clk::now();
    if (m == 0) H.cond_max = fit.cond_max;
    PackRows rows;
    rows.W = 15;
    rows.regular = fit.regular;
    const int n2 = (int)fit.irr.size();
    std::vector<int> order(n2);
    for (int r = 0; r < n2; ++r) order[r] = r;
    if (m < nl - 1 && n2) {
      // renumber the fitted rows into the boundary order of Alg. 3
      PackRows tmp;
      tmp.irr = fit.irr;
      order = boundary_order(cg, tmp);
    }
    for (int r : order) {
      rows.irr.push_back(fit.irr[r]);
      for (int k = 0; k < 15; ++k) {
        rows.cols.push_back(fit.cols[r][k]);
        rows.beta.push_back(fit.beta[r][k]);
      }
      rows.nb.push_back(fit.nb[r]);
      rows.seg.push_back(fit.seg[r]);
    }
    rc = pack_level(cg, rows, par, m == nl - 1, m == 0, H.levels[m], err);
    H.ms_blocks += ms_since(t0);
    if (rc) return rc;
    H.rows.push_back(std::move(rows));
    if (m == 0) H.nseg = (int)cg.segs.size();
    if (m == nl - 1) {
      t0 = clk::now();
      rc = finish_bottom(H.levels[m], cg, w, err);
      H.ms_bottom += ms_since(t0);
      if (rc) return rc;
    }
  }
  return CCM_OK;
}

int build_transposed(const Hierarchy& H, const ccm_params& par, Hierarchy& T, std::string& err) {
  T.a = H.a;
  T.b = H.b;
  T.c = H.c;
  T.nseg = 0;
  T.cond_max = H.cond_max;
  const int nl = (int)H.levels.size();
  T.levels.resize(nl);
  double w[5][5];
  regular_stencil(H.a, H.b, H.c, w);
  for (int m = 0; m < nl; ++m) {
    const CutLevel& cg = H.cut[m];
    PackRows t = transpose_rows(cg, H.rows[m], w);
    if (m < nl - 1 && !t.irr.empty()) {
      std::vector<int> order = boundary_order(cg, t);
      PackRows p;
      p.W = t.W;
      p.regular.swap(t.regular);
      for (int r : order) {
        p.irr.push_back(t.irr[r]);
        for (int k = 0; k < t.W; ++k) {
          p.cols.push_back(t.cols[(long)r * t.W + k]);
          p.beta.push_back(t.beta[(long)r * t.W + k]);
        }
        p.nb.push_back(0.0);
        p.seg.push_back(-1);
      }
      t = std::move(p);
    }
    int rc = pack_level(cg, t, par, m == nl - 1, false, T.levels[m], err);
    if (rc) return rc;
    if (m == nl - 1) {
      rc = finish_bottom(T.levels[m], cg, w, err);
      if (rc) return rc;
    }
  }
  return CCM_OK;
}

}  // namespace ccm
