// Regular stencils, PLG stencils and weighted minimum-norm fits (Sec. 3.2 - 3.4).
//
// Regular cells (every cell of the 5x5 box pure) use eq. stdLap in x1 and x2 and the
// product of eq. stdGrad for the cross term.  Every other non-empty cell gets a fitted row:
// among poised 15-cell lattices near the cell (5 parallel grid lines carrying 5, 4, 3, 2, 1
// cells -- a transformed principal lattice, poised for Pi_4) the first NCAND by integer cost
// sum |j_k - i|^2 are fitted with beta = W M^T (M W M^T)^-1 L (eq. derivedCoefAgain, weights
// eq. weightDef, basis ((x - p)/h)^alpha recentred at the stencil's bounding-box centre),
// and the lattice whose coefficients have the least weighted norm ||beta||_{W^-1} is kept.
// Coefficients are stored h^2-scaled (the discrete equation is multiplied by h^2).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <thread>

#include "host.h"

namespace ccm {

static const int RADII[3] = {3, 4, 5};
static const int NCAND = 12;

// scale of the Robin boundary column, |gamma1| + |gamma2| / h
static double robin_norm(double g1, double g2, double h) { return std::fabs(g1) + std::fabs(g2) / h; }

void regular_stencil(double a, double b, double c, double w[5][5]) {
  static const double lap[5] = {-1.0, 16.0, -30.0, 16.0, -1.0};
  static const double grad[5] = {1.0, -8.0, 0.0, 8.0, -1.0};
  for (int dj = 0; dj < 5; ++dj)
    for (int di = 0; di < 5; ++di) w[dj][di] = 0.0;
  for (int m = 0; m < 5; ++m) {
    w[2][m] += a * lap[m] / 12.0;
    w[m][2] += c * lap[m] / 12.0;
  }
  if (b != 0.0)
    for (int dj = 0; dj < 5; ++dj)
      for (int di = 0; di < 5; ++di) w[dj][di] += b * grad[di] * grad[dj] / 144.0;
}

namespace {

struct Perms {
  int p[120][5];
  Perms() {
    int a[5] = {1, 2, 3, 4, 5}, n = 0;
    do {
      for (int k = 0; k < 5; ++k) p[n][k] = a[k];
      ++n;
    } while (std::next_permutation(a, a + 5));
  }
};
const Perms& perms() {
  static Perms P;
  return P;
}

struct Cand {
  long cost;
  int o, si, pk;
};

// Up to NCAND candidate lattices around cell (i, j), best first.
bool plg_candidates(const CutLevel& cg, int i, int j, std::vector<std::array<int, 15>>& out) {
  const Perms& P = perms();
  out.clear();
  for (int R : RADII) {
    const int W = 2 * R + 1;
    std::vector<Cand> found;
    std::vector<int> lines_du[2][11];
    std::vector<std::array<int, 5>> subs;
    {
      std::vector<int> others;
      for (int dv = -R; dv <= R; ++dv)
        if (dv != 0) others.push_back(dv);
      int n = (int)others.size();
      for (int a = 0; a < n; ++a)
        for (int b = a + 1; b < n; ++b)
          for (int c = b + 1; c < n; ++c)
            for (int d = c + 1; d < n; ++d) {
              std::array<int, 5> s = {others[a], others[b], others[c], others[d], 0};
              std::sort(s.begin(), s.end());
              subs.push_back(s);
            }
    }
    for (int o = 0; o < 2; ++o) {
      long tab[11][5];
      for (int dv = -R; dv <= R; ++dv) {
        std::vector<int>& av = lines_du[o][dv + R];
        av.clear();
        for (int du = -R; du <= R; ++du) {
          int ii = o == 0 ? i + du : i + dv, jj = o == 0 ? j + dv : j + du;
          if (ii >= 0 && ii < cg.nx && jj >= 0 && jj < cg.ny && cg.status[(long)jj * cg.nx + ii] != ST_EMPTY)
            av.push_back(du);
        }
        std::sort(av.begin(), av.end(), [](int x, int y) {
          if (x * x != y * y) return x * x < y * y;
          return x < y;
        });
        long acc = 0;
        for (int m = 1; m <= 5; ++m) {
          if ((int)av.size() >= m) {
            acc += (long)av[m - 1] * av[m - 1];
            tab[dv + R][m - 1] = acc + (long)m * dv * dv;
          } else {
            tab[dv + R][m - 1] = -1;
          }
        }
      }
      for (int si = 0; si < (int)subs.size(); ++si) {
        for (int pk = 0; pk < 120; ++pk) {
          long cost = 0;
          bool ok = true;
          for (int l = 0; l < 5; ++l) {
            long v = tab[subs[si][l] + R][P.p[pk][l] - 1];
            if (v < 0) { ok = false; break; }
            cost += v;
          }
          if (ok) found.push_back({cost, o, si, pk});
        }
      }
    }
    (void)W;
    if (found.empty()) continue;
    // the first NCAND candidates in the total order (cost, orientation, subset, counts); the
    // order has no ties, so a partial sort gives the same leaders as a full sort
    int nk = std::min<int>(NCAND, (int)found.size());
    std::partial_sort(found.begin(), found.begin() + nk, found.end(), [](const Cand& x, const Cand& y) {
      if (x.cost != y.cost) return x.cost < y.cost;
      if (x.o != y.o) return x.o < y.o;
      if (x.si != y.si) return x.si < y.si;
      return x.pk < y.pk;
    });
    for (int k = 0; k < nk; ++k) {
      const Cand& c = found[k];
      std::vector<std::pair<int, int>> cells;   // (dx, dy)
      for (int l = 0; l < 5; ++l) {
        int dv = subs[c.si][l], m = P.p[c.pk][l];
        const std::vector<int>& av = lines_du[c.o][dv + R];
        for (int q = 0; q < m; ++q) {
          int du = av[q];
          if (c.o == 0) cells.push_back({du, dv});
          else cells.push_back({dv, du});
        }
      }
      std::stable_sort(cells.begin(), cells.end(), [](const std::pair<int, int>& x, const std::pair<int, int>& y) {
        bool xi = (x.first == 0 && x.second == 0), yi = (y.first == 0 && y.second == 0);
        if (xi != yi) return xi;
        if (x.second != y.second) return x.second < y.second;
        return x.first < y.first;
      });
      std::array<int, 15> lin;
      for (int q = 0; q < 15; ++q) lin[q] = (j + cells[q].second) * cg.nx + (i + cells[q].first);
      out.push_back(lin);
    }
    return true;
  }
  return false;
}

// Solve the SPD system A x = b (n <= 16) by Cholesky; false if not positive definite.
bool chol_solve(double* A, int n, double* b) {
  for (int k = 0; k < n; ++k) {
    double d = A[k * n + k];
    for (int m = 0; m < k; ++m) d -= A[k * n + m] * A[k * n + m];
    if (!(d > 0.0)) return false;
    d = std::sqrt(d);
    A[k * n + k] = d;
    for (int r = k + 1; r < n; ++r) {
      double s = A[r * n + k];
      for (int m = 0; m < k; ++m) s -= A[r * n + m] * A[k * n + m];
      A[r * n + k] = s / d;
    }
  }
  for (int r = 0; r < n; ++r) {
    double s = b[r];
    for (int m = 0; m < r; ++m) s -= A[r * n + m] * b[m];
    b[r] = s / A[r * n + r];
  }
  for (int r = n - 1; r >= 0; --r) {
    double s = b[r];
    for (int m = r + 1; m < n; ++m) s -= A[m * n + r] * b[m];
    b[r] = s / A[r * n + r];
  }
  return true;
}

// 2-norm condition number of a 15x15 matrix by one-sided Jacobi.
double cond2(const double M[15][15]) {
  double U[15][15];
  for (int r = 0; r < 15; ++r)
    for (int c = 0; c < 15; ++c) U[r][c] = M[r][c];
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0;
    for (int p = 0; p < 15; ++p)
      for (int q = p + 1; q < 15; ++q) {
        double a = 0, b = 0, g = 0;
        for (int r = 0; r < 15; ++r) {
          a += U[r][p] * U[r][p];
          b += U[r][q] * U[r][q];
          g += U[r][p] * U[r][q];
        }
        if (std::fabs(g) <= 1e-300 || std::fabs(g) <= 1e-15 * std::sqrt(a * b)) continue;
        off = std::max(off, std::fabs(g) / std::sqrt(a * b));
        double zeta = (b - a) / (2 * g);
        double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1 + zeta * zeta));
        double cs = 1 / std::sqrt(1 + t * t), sn = cs * t;
        for (int r = 0; r < 15; ++r) {
          double up = U[r][p], uq = U[r][q];
          U[r][p] = cs * up - sn * uq;
          U[r][q] = sn * up + cs * uq;
        }
      }
    if (off < 1e-15) break;
  }
  double smax = 0, smin = 1e300;
  for (int c = 0; c < 15; ++c) {
    double s = 0;
    for (int r = 0; r < 15; ++r) s += U[r][c] * U[r][c];
    s = std::sqrt(s);
    smax = std::max(smax, s);
    smin = std::min(smin, s);
  }
  return smin > 0 ? smax / smin : 1e300;
}

struct FitOut {
  double beta[16];
  double norm;
  double M15[15][15];
  bool ok;
};

void fit(const CutLevel& cg, int i, int j, const std::array<int, 15>& cells, double a, double b, double c,
         FitOut& fo) {
  const int nx = cg.nx;
  const long lin = (long)j * nx + i;
  int imin = 1 << 30, imax = -(1 << 30), jmin = 1 << 30, jmax = -(1 << 30);
  for (int q = 0; q < 15; ++q) {
    int ci = cells[q] % nx, cj = cells[q] / nx;
    imin = std::min(imin, ci);
    imax = std::max(imax, ci);
    jmin = std::min(jmin, cj);
    jmax = std::max(jmax, cj);
  }
  // frame offsets of a cell centre from p, in units of h (half-integers)
  const double pxi = 0.5 * (imin + imax), pyj = 0.5 * (jmin + jmax);
  double M[15][16];
  for (int q = 0; q < 15; ++q) {
    int ci = cells[q] % nx, cj = cells[q] / nx;
    Mom m = shift_moments(cg.moments(cells[q]), ci - pxi, cj - pyj);
    double v = cg.vol[cells[q]];
    for (int k = 0; k < NMOM; ++k) M[k][q] = m[k] / v;
  }
  for (int r = 0; r < 15; ++r)
    for (int q = 0; q < 15; ++q) fo.M15[r][q] = M[r][q];
  const double dx = i - pxi, dy = j - pyj;
  Mom mi = shift_moments(cg.moments((int)lin), dx, dy);
  double vi = cg.vol[lin];
  double Lhat[15];
  for (int k = 0; k < NMOM; ++k) {
    int p = mono_p(k), q = mono_q(k);
    double v = 0;
    if (p >= 2) v += a * p * (p - 1) * mi[mono_index(p - 2, q)];
    if (p >= 1 && q >= 1) v += b * p * q * mi[mono_index(p - 1, q - 1)];
    if (q >= 2) v += c * q * (q - 1) * mi[mono_index(p, q - 2)];
    Lhat[k] = v / vi;
  }
  double w[16];
  for (int q = 0; q < 15; ++q) {
    int ci = cells[q] % nx, cj = cells[q] / nx;
    w[q] = std::max(std::hypot((double)(ci - i), (double)(cj - j)), 0.5);
  }
  int ncol = 15;
  auto sit = cg.seg_of.find((int)lin);
  if (sit != cg.seg_of.end()) {
    int s = sit->second;
    double S = cg.bm0[s][0];
    // the boundary column <N phi_k> in the scaled frame: the average of the monomial
    // (Dirichlet), of its normal derivative (Neumann), or gamma1 times the first plus gamma2 / h
    // times the second, divided by |gamma1| + |gamma2| / h (Robin), so that the Robin column
    // reduces to the other two when a coefficient vanishes
    double cd[NMOM], cn[NMOM];
    const int bc = cg.seg_bc[s];
    if (bc != CCM_NEUMANN) {
      Mom g = shift_moments(cg.bm0[s], dx, dy);
      for (int k = 0; k < NMOM; ++k) cd[k] = g[k] / S;
    }
    if (bc != CCM_DIRICHLET) {
      Mom gx = shift_moments(cg.bmx[s], dx, dy), gy = shift_moments(cg.bmy[s], dx, dy);
      for (int k = 0; k < NMOM; ++k) {
        int p = mono_p(k), q = mono_q(k);
        double v = 0;
        if (p >= 1) v += p * gx[mono_index(p - 1, q)];
        if (q >= 1) v += q * gy[mono_index(p, q - 1)];
        cn[k] = v / S;
      }
    }
    for (int k = 0; k < NMOM; ++k) {
      if (bc == CCM_DIRICHLET) M[k][15] = cd[k];
      else if (bc == CCM_NEUMANN) M[k][15] = cn[k];
      else {
        const double g1 = cg.seg_gamma[s][0], g2 = cg.seg_gamma[s][1];
        M[k][15] = (g1 * cd[k] + (g2 / cg.h) * cn[k]) / robin_norm(g1, g2, cg.h);
      }
    }
    w[15] = 0.5;
    ncol = 16;
  }
  // (M W M^T) y = Lhat, beta = W M^T y with W = diag(1/w)
  double A[15 * 15], y[15];
  for (int r = 0; r < 15; ++r) {
    for (int s = 0; s <= r; ++s) {
      double acc = 0;
      for (int q = 0; q < ncol; ++q) acc += M[r][q] * M[s][q] / w[q];
      A[r * 15 + s] = acc;
      A[s * 15 + r] = acc;
    }
    y[r] = Lhat[r];
  }
  fo.ok = chol_solve(A, 15, y);
  double nrm = 0;
  for (int q = 0; q < 16; ++q) fo.beta[q] = 0;
  for (int q = 0; q < ncol; ++q) {
    double acc = 0;
    for (int r = 0; r < 15; ++r) acc += M[r][q] * y[r];
    fo.beta[q] = acc / w[q];
    nrm += w[q] * fo.beta[q] * fo.beta[q];
  }
  fo.norm = nrm;
}

}  // namespace

int discretize_level(const CutLevel& cg, double a, double b, double c, int nthreads, Rows& rows,
                     std::string& err, FitBatcher* fb) {
  const int nx = cg.nx, ny = cg.ny;
  const long N = (long)nx * ny;
  rows.regular.assign(N, 0);
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      long q = (long)j * nx + i;
      if (cg.status[q] == ST_EMPTY) continue;
      bool reg = true;
      for (int dj = -2; dj <= 2 && reg; ++dj)
        for (int di = -2; di <= 2; ++di) {
          int ii = i + di, jj = j + dj;
          if (ii < 0 || ii >= nx || jj < 0 || jj >= ny || cg.status[(long)jj * nx + ii] != ST_PURE) {
            reg = false;
            break;
          }
        }
      rows.regular[q] = reg ? 1 : 0;
    }
  rows.irr.clear();
  for (long q = 0; q < N; ++q)
    if (cg.status[q] != ST_EMPTY && !rows.regular[q]) rows.irr.push_back((int)q);
  const size_t n2 = rows.irr.size();
  rows.cols.assign(n2, {});
  rows.beta.assign(n2, {});
  rows.nb.assign(n2, 0.0);
  rows.seg.assign(n2, -1);
  std::vector<double> conds(n2, 0.0);
  std::atomic<int> status{CCM_OK};
  std::atomic<size_t> next{0};
  int nt = nthreads > 0 ? nthreads : (int)std::max(1u, std::thread::hardware_concurrency());
  nt = std::min<int>(nt, std::max<size_t>(1, n2 / 16 + 1));
  // N g enters the scaled rows (h^2 L) with the column's scale undone: h^0 (Dirichlet),
  // h (Neumann), 1 / (|gamma1| + |gamma2| / h) (Robin)
  auto set_boundary = [&](size_t r, int lin, double b15) {
    auto sit = cg.seg_of.find(lin);
    if (sit == cg.seg_of.end()) return;
    const int s = sit->second, bc = cg.seg_bc[s];
    rows.seg[r] = s;
    rows.nb[r] = bc == CCM_DIRICHLET ? b15
                 : bc == CCM_NEUMANN ? b15 * cg.h
                                     : b15 / robin_norm(cg.seg_gamma[s][0], cg.seg_gamma[s][1], cg.h);
  };
  if (fb && n2 > 0) {
    // candidates of every row on the host threads, all fits in one batch, the same choice
    std::vector<std::vector<std::array<int, 15>>> cands(n2);
    std::vector<std::thread> th;
    for (int t = 0; t < nt; ++t)
      th.emplace_back([&]() {
        while (true) {
          const size_t r = next.fetch_add(1);
          if (r >= n2 || status.load() != CCM_OK) break;
          const int lin = rows.irr[r];
          if (!plg_candidates(cg, lin % nx, lin / nx, cands[r])) status.store(CCM_EPLG);
        }
      });
    for (auto& t : th) t.join();
    if (status.load() != CCM_OK) {
      err = "no poised PLG stencil within radius 5";
      return CCM_EPLG;
    }
    std::vector<size_t> first(n2 + 1, 0);
    for (size_t r = 0; r < n2; ++r) first[r + 1] = first[r] + cands[r].size();
    std::vector<int32_t> prow(first[n2]);
    std::vector<std::array<int, 15>> pc(first[n2]);
    for (size_t r = 0; r < n2; ++r)
      for (size_t k = 0; k < cands[r].size(); ++k) {
        prow[first[r] + k] = rows.irr[r];
        pc[first[r] + k] = cands[r][k];
      }
    std::vector<double> beta, norm;
    std::vector<uint8_t> ok;
    int rc = fb->fit(cg, a, b, c, prow, pc, beta, norm, ok);
    if (rc) {
      err = "device fits failed";
      return rc;
    }
    std::vector<int32_t> crow(n2);
    std::vector<std::array<int, 15>> chosen(n2);
    for (size_t r = 0; r < n2; ++r) {
      long bk = -1;
      for (size_t k = first[r]; k < first[r + 1]; ++k) {
        if (!ok[k]) continue;
        if (bk < 0 || norm[k] < norm[bk] * (1.0 - 1e-9)) bk = (long)k;
      }
      if (bk < 0) {
        err = "singular weighted normal equations";
        return CCM_ESINGULAR;
      }
      rows.cols[r] = pc[bk];
      for (int q = 0; q < 15; ++q) rows.beta[r][q] = beta[16 * bk + q];
      set_boundary(r, rows.irr[r], beta[16 * bk + 15]);
      crow[r] = rows.irr[r];
      chosen[r] = pc[bk];
    }
    rc = fb->cond(cg, crow, chosen, conds);
    if (rc) {
      err = "device fits failed";
      return rc;
    }
    rows.cond_max = 0;
    for (double v : conds) rows.cond_max = std::max(rows.cond_max, v);
    return CCM_OK;
  }
  auto worker = [&]() {
    std::vector<std::array<int, 15>> cands;
    FitOut fo, best;
    while (true) {
      size_t r = next.fetch_add(1);
      if (r >= n2 || status.load() != CCM_OK) break;
      int lin = rows.irr[r], i = lin % nx, j = lin / nx;
      if (!plg_candidates(cg, i, j, cands)) {
        status.store(CCM_EPLG);
        break;
      }
      int bk = -1;
      for (size_t k = 0; k < cands.size(); ++k) {
        fit(cg, i, j, cands[k], a, b, c, fo);
        if (!fo.ok) continue;
        if (bk < 0 || fo.norm < best.norm * (1.0 - 1e-9)) {
          best = fo;
          bk = (int)k;
        }
      }
      if (bk < 0) {
        status.store(CCM_ESINGULAR);
        break;
      }
      rows.cols[r] = cands[bk];
      for (int q = 0; q < 15; ++q) rows.beta[r][q] = best.beta[q];
      set_boundary(r, lin, best.beta[15]);
      conds[r] = cond2(best.M15);
    }
  };
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t) th.emplace_back(worker);
  for (auto& t : th) t.join();
  if (status.load() != CCM_OK) {
    err = status.load() == CCM_EPLG ? "no poised PLG stencil within radius 5" : "singular weighted normal equations";
    return status.load();
  }
  rows.cond_max = 0;
  for (double v : conds) rows.cond_max = std::max(rows.cond_max, v);
  return CCM_OK;
}

}  // namespace ccm
