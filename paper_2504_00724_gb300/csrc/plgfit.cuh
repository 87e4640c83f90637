// Device side of the setup's fits (Sec. 3.3): the weighted least-squares coefficients of
// many (fitted row, candidate PLG stencil) pairs at once, and the 2-norm condition number of
// the FV sample matrix of a chosen stencil.  One warp per pair, the 15 x 16 sample matrix in
// shared memory.  The arithmetic is that of the host fit (eq. derivedCoefAgain: the FV sample
// matrix M of the basis x^p y^q, p + q <= 4, in the frame centred on the stencil's bounding
// box; L_hat the operator applied to the basis over the cell; the boundary column of the
// cell's boundary operator; W = diag(1/w), w from eq. weightDef; beta = W M^T (M W M^T)^-1
// L_hat) in another summation order, so the two agree to rounding.
#pragma once

#include <cstdint>

namespace ccm {
namespace dev {

constexpr int FNM = 15;           // monomials of degree <= 4

struct FitLevel {
  int nx;
  double h, a, b, c;
  const double* mom;              // [nm][15] moments of the cut cells (own frame, units of h)
  const double* vol;              // [nm] their volumes / h^2
  const int32_t* seg_bc;          // [nseg]
  const double* seg_mom;          // [nseg][3][15]: <1>, <n_x>, <n_y> moments of the boundary piece
  const double* seg_gamma;        // [nseg][2]
  double pure[FNM];               // moments of a pure cell
};

struct FitBatch {
  int n;                          // pairs
  const int32_t* row;             // [n][4]: cell i, j, moment id (-1: pure), segment (-1: none)
  const int32_t* cells;           // [n][15][2]: linear index, moment id (-1: pure)
  double* beta;                   // [n][16]
  double* norm;                   // [n]
  uint8_t* ok;                    // [n]
  double* cond;                   // [n] (cond mode)
};

__device__ __forceinline__ int fmono_p(int k) {
  const int d = k < 1 ? 0 : k < 3 ? 1 : k < 6 ? 2 : k < 10 ? 3 : 4;
  return d - (k - d * (d + 1) / 2);
}
__device__ __forceinline__ int fmono_q(int k) {
  const int d = k < 1 ? 0 : k < 3 ? 1 : k < 6 ? 2 : k < 10 ? 3 : 4;
  return k - d * (d + 1) / 2;
}
__device__ __forceinline__ int fmono_index(int p, int q) {
  const int d = p + q;
  return d * (d + 1) / 2 + q;
}
__device__ __forceinline__ double fbinom(int n, int k) {
  // n <= 4
  const double t[5][5] = {{1, 0, 0, 0, 0}, {1, 1, 0, 0, 0}, {1, 2, 1, 0, 0}, {1, 3, 3, 1, 0}, {1, 4, 6, 4, 1}};
  return t[n][k];
}

// moment k of m shifted by (dx, dy): the integral of (x + dx)^p (y + dy)^q from the moments
// of x^a y^b
__device__ __forceinline__ double fshift(const double* m, int k, double dx, double dy) {
  const int p = fmono_p(k), q = fmono_q(k);
  double px[5], py[5];
  px[0] = 1;
  py[0] = 1;
#pragma unroll
  for (int e = 1; e < 5; ++e) {
    px[e] = px[e - 1] * dx;
    py[e] = py[e - 1] * dy;
  }
  double s = 0;
  for (int a = 0; a <= p; ++a)
    for (int b = 0; b <= q; ++b) s += fbinom(p, a) * fbinom(q, b) * px[p - a] * py[q - b] * m[fmono_index(a, b)];
  return s;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

struct FitSmem {
  double M[FNM][17];              // columns 0..14 stencil cells, 15 the boundary column
  double A[FNM][FNM + 1];
  double Lh[FNM];
  double y[FNM];
  double w[16];
  double wi[16];                  // 1 / w
};

// frame of a pair: the centre of the stencil's bounding box (half-integer cell units)
__device__ __forceinline__ void fit_frame(const FitLevel& L, const int32_t* cells, int lane, double& pxi, double& pyj) {
  int lin = lane < FNM ? cells[2 * lane] : cells[0];
  int ci = lin % L.nx, cj = lin / L.nx;
  int imin = ci, imax = ci, jmin = cj, jmax = cj;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    imin = min(imin, __shfl_xor_sync(0xffffffffu, imin, o));
    imax = max(imax, __shfl_xor_sync(0xffffffffu, imax, o));
    jmin = min(jmin, __shfl_xor_sync(0xffffffffu, jmin, o));
    jmax = max(jmax, __shfl_xor_sync(0xffffffffu, jmax, o));
  }
  pxi = 0.5 * (imin + imax);
  pyj = 0.5 * (jmin + jmax);
}

// the 15 x 15 FV sample matrix into S.M (lane q builds column q)
__device__ __forceinline__ void fit_sample(const FitLevel& L, const int32_t* cells, int lane, double pxi, double pyj,
                                           FitSmem& S) {
  if (lane < FNM) {
    const int lin = cells[2 * lane], id = cells[2 * lane + 1];
    const int ci = lin % L.nx, cj = lin / L.nx;
    const double* m = id < 0 ? L.pure : L.mom + (long)id * FNM;
    const double v = id < 0 ? 1.0 : L.vol[id];
    for (int k = 0; k < FNM; ++k) S.M[k][lane] = fshift(m, k, ci - pxi, cj - pyj) / v;
  }
}

__global__ void __launch_bounds__(128) k_plg_fit(FitLevel L, FitBatch B) {
  __shared__ FitSmem sm[4];
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const int pair = blockIdx.x * 4 + wi;
  if (pair >= B.n) return;               // whole warps leave together
  FitSmem& S = sm[wi];
  const int32_t* rw = B.row + 4 * (long)pair;
  const int32_t* cells = B.cells + 30 * (long)pair;
  const int i = rw[0], j = rw[1], rid = rw[2], seg = rw[3];
  double pxi, pyj;
  fit_frame(L, cells, lane, pxi, pyj);
  fit_sample(L, cells, lane, pxi, pyj, S);
  const double dx = i - pxi, dy = j - pyj;
  const int ncol = seg >= 0 ? 16 : 15;
  if (lane == FNM && seg >= 0) {
    // the boundary column <N phi_k> (scaled frame)
    const double* g0 = L.seg_mom + (long)seg * 3 * FNM;
    const double Sl = g0[0];
    const int bc = L.seg_bc[seg];
    const double g1 = L.seg_gamma[2 * seg], g2 = L.seg_gamma[2 * seg + 1];
    const double rn = fabs(g1) + fabs(g2) / L.h;
    for (int k = 0; k < FNM; ++k) {
      const int p = fmono_p(k), q = fmono_q(k);
      double cd = 0, cn = 0;
      if (bc != 2) cd = fshift(g0, k, dx, dy) / Sl;
      if (bc != 1) {
        double v = 0;
        if (p >= 1) v += p * fshift(g0 + FNM, fmono_index(p - 1, q), dx, dy);
        if (q >= 1) v += q * fshift(g0 + 2 * FNM, fmono_index(p, q - 1), dx, dy);
        cn = v / Sl;
      }
      S.M[k][15] = bc == 1 ? cd : bc == 2 ? cn : (g1 * cd + (g2 / L.h) * cn) / rn;
    }
  }
  if (lane == 16) {
    // L_hat_k = <L phi_k> over the row's cell
    const double* m = rid < 0 ? L.pure : L.mom + (long)rid * FNM;
    const double vi = rid < 0 ? 1.0 : L.vol[rid];
    for (int k = 0; k < FNM; ++k) {
      const int p = fmono_p(k), q = fmono_q(k);
      double v = 0;
      if (p >= 2) v += L.a * p * (p - 1) * fshift(m, fmono_index(p - 2, q), dx, dy);
      if (p >= 1 && q >= 1) v += L.b * p * q * fshift(m, fmono_index(p - 1, q - 1), dx, dy);
      if (q >= 2) v += L.c * q * (q - 1) * fshift(m, fmono_index(p, q - 2), dx, dy);
      S.Lh[k] = v / vi;
    }
  }
  if (lane < FNM) {
    const int lin = cells[2 * lane];
    const int ci = lin % L.nx, cj = lin / L.nx;
    S.w[lane] = fmax(hypot((double)(ci - i), (double)(cj - j)), 0.5);
    S.wi[lane] = 1.0 / S.w[lane];
  }
  if (lane == FNM) {
    S.w[15] = 0.5;
    S.wi[15] = 2.0;
  }
  __syncwarp();
  // A = M W M^T (lower triangle, 120 entries over the lanes), W = diag(1 / w)
  for (int e = lane; e < 120; e += 32) {
    int r = 0;
    while ((r + 1) * (r + 2) / 2 <= e) ++r;
    const int s = e - r * (r + 1) / 2;
    double acc = 0;
    for (int q = 0; q < ncol; ++q) acc += S.M[r][q] * S.M[s][q] * S.wi[q];
    S.A[r][s] = acc;
  }
  __syncwarp();
  // Cholesky (left-looking by columns) and the two triangular solves
  bool ok = true;
  for (int k = 0; k < FNM; ++k) {
    double d = S.A[k][k];
    for (int m = 0; m < k; ++m) d -= S.A[k][m] * S.A[k][m];
    if (!(d > 0.0)) {
      ok = false;
      break;
    }
    d = sqrt(d);
    const int r = k + 1 + lane;
    double v = 0;
    if (r < FNM) {
      v = S.A[r][k];
      for (int m = 0; m < k; ++m) v -= S.A[r][m] * S.A[k][m];
    }
    __syncwarp();
    if (r < FNM) S.A[r][k] = v / d;
    if (lane == 0) S.A[k][k] = d;
    __syncwarp();
  }
  if (!ok) {
    if (lane == 0) B.ok[pair] = 0;
    return;
  }
  // the two triangular solves with the Cholesky factor, column by column: once y_r is known,
  // lane m subtracts its term from its own partial sum
  {
    double v = lane < FNM ? S.Lh[lane] : 0.0;
    for (int r = 0; r < FNM; ++r) {
      const double yr = __shfl_sync(0xffffffffu, v, r) / S.A[r][r];
      if (lane == r) v = yr;
      else if (lane > r && lane < FNM) v -= S.A[lane][r] * yr;
    }
    for (int r = FNM - 1; r >= 0; --r) {
      const double yr = __shfl_sync(0xffffffffu, v, r) / S.A[r][r];
      if (lane == r) v = yr;
      else if (lane < r) v -= S.A[r][lane] * yr;
    }
    if (lane < FNM) S.y[lane] = v;
  }
  __syncwarp();
  double bq = 0, nq = 0;
  if (lane < ncol) {
    double acc = 0;
    for (int r = 0; r < FNM; ++r) acc += S.M[r][lane] * S.y[r];
    bq = acc * S.wi[lane];
    nq = S.w[lane] * bq * bq;
  }
  const double nrm = warp_sum(nq);
  if (lane < 16) B.beta[16 * (long)pair + lane] = lane < ncol ? bq : 0.0;
  if (lane == 0) {
    B.norm[pair] = nrm;
    B.ok[pair] = 1;
  }
}

// 2-norm condition number of the 15 x 15 FV sample matrix of each pair by one-sided Jacobi
// (column rotations until every pair of columns is orthogonal to 1e-15); lane r samples row
// r, lanes 1..7 then rotate seven disjoint column pairs at a time
__global__ void __launch_bounds__(128) k_plg_cond(FitLevel L, FitBatch B) {
  __shared__ FitSmem sm[4];
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const int pair = blockIdx.x * 4 + wi;
  if (pair >= B.n) return;
  FitSmem& S = sm[wi];
  const int32_t* cells = B.cells + 30 * (long)pair;
  double pxi, pyj;
  fit_frame(L, cells, lane, pxi, pyj);
  fit_sample(L, cells, lane, pxi, pyj, S);
  __syncwarp();
  // parallel cyclic ordering: a round robin over 16 players (player 15 a dummy) pairs the
  // columns (s + k) mod 15 and (s - k) mod 15, k = 1..7, in step s; those pairs are disjoint,
  // so lanes 1..7 rotate them at once, and the 15 steps of a sweep visit every pair once
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0;
    for (int st = 0; st < FNM; ++st) {
      if (lane >= 1 && lane <= 7) {
        int p = (st + lane) % FNM, q = (st + FNM - lane) % FNM;
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        double a = 0, b = 0, g = 0;
        for (int r = 0; r < FNM; ++r) {
          const double up = S.M[r][p], uq = S.M[r][q];
          a += up * up;
          b += uq * uq;
          g += up * uq;
        }
        if (!(fabs(g) <= 1e-300 || fabs(g) <= 1e-15 * sqrt(a * b))) {
          off = fmax(off, fabs(g) / sqrt(a * b));
          const double zeta = (b - a) / (2 * g);
          const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1 + zeta * zeta));
          const double cs = 1 / sqrt(1 + t * t), sn = cs * t;
          for (int r = 0; r < FNM; ++r) {
            const double up = S.M[r][p], uq = S.M[r][q];
            S.M[r][p] = cs * up - sn * uq;
            S.M[r][q] = sn * up + cs * uq;
          }
        }
      }
      __syncwarp();
    }
    for (int o = 16; o; o >>= 1) off = fmax(off, __shfl_xor_sync(0xffffffffu, off, o));
    if (off < 1e-15) break;
  }
  double smax = 0, smin = 1e300;
  for (int c = 0; c < FNM; ++c) {
    const double u = lane < FNM ? S.M[lane][c] : 0.0;
    const double s = sqrt(warp_sum(u * u));
    smax = fmax(smax, s);
    smin = fmin(smin, s);
  }
  if (lane == 0) B.cond[pair] = smin > 0 ? smax / smin : 1e300;
}

}  // namespace dev
}  // namespace ccm
