// Krylov acceleration of the mixed-precision outer iteration: the correction e of one outer
// step, which plain iterative refinement takes as e = M r (M = inner_cycles FP32 V-cycles of
// Alg. 2 from a zero guess), is instead the GMRES(m) solution of L e = r with M as a right
// preconditioner: e = Z y with z_j = M v_j, the v_j an orthonormal basis of the Krylov space
// of L M built by classical Gram-Schmidt with one re-orthogonalisation, and y minimising
// || beta e_1 - H y ||_2 over the (m + 1) x m Hessenberg matrix H.  Everything inside the step
// is FP32 on level 0 (vectors, the operator, the preconditioner) with FP64 dot products; the
// FP64 residual r_hat - L u_hat around it is unchanged, so the refinement still converges to
// the FP64 solution (GMRES-based iterative refinement).
//
// Vectors are padded level-0 arrays; only non-empty cells are ever written, so empty cells
// stay zero and the reductions may run over whole 32 x 8 tiles.  Every reduction is two
// launches: per-CTA partial sums in FP64, then one CTA that adds them in a fixed order, so the
// results do not depend on scheduling.  Nothing here synchronises with the host: the scalars
// (Gram-Schmidt coefficients, H, y) stay in device memory and the step is captured into the
// outer iteration's graph.
#pragma once

#include "kernels.cuh"

namespace ccm {
namespace dev {

constexpr int KRY_MAXM = 8;          // largest GMRES restart length
constexpr int KRY_GRID = 304;        // CTAs of the partial-sum kernels
constexpr int KRY_THREADS = 256;     // = one 32 x 8 tile per CTA step

struct KryVecs {
  const float* v[KRY_MAXM + 1];
};

// scalars of one GMRES step (device memory)
struct KryScalars {
  double part[(KRY_MAXM + 1) * KRY_GRID];   // per-CTA partial sums [vector][cta]
  double c[KRY_MAXM + 1];                   // coefficients of the last reduction
  double H[(KRY_MAXM + 1) * KRY_MAXM];      // Hessenberg matrix, column-major, leading dim m + 1
  double beta;                              // || r ||_2 at the start of the step
  double y[KRY_MAXM];                       // least-squares solution
};

// Vector kernels run persistent over the 32 x 8 tiles that hold a non-empty cell (one cell
// per thread per tile), in FP32 arithmetic: GB300 issues FP64 at 1/64 of the FP32 rate, so only
// the per-thread sums of the reductions leave FP32, compensated (Neumaier) until then.
struct Comp {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float t = s + x;
    c += fabsf(s) >= fabsf(x) ? (s - t) + x : (x - t) + s;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

__device__ __forceinline__ bool kcell(const int32_t* __restrict__ tiles, int t, int nx, int ny, int pitch, long& p) {
  const int ci = tiles[2 * t] * TX + (threadIdx.x & 31), cj = tiles[2 * t + 1] * TY + (threadIdx.x >> 5);
  p = (long)(cj + 2) * pitch + (ci + 2);
  return ci < nx && cj < ny;
}

// per-CTA partial sums of acc[0 .. n) into part[i][blockIdx.x] (FP64 across the CTA)
__device__ __forceinline__ void kpartials(const Comp (&acc)[KRY_MAXM + 1], int n, KryScalars* __restrict__ S) {
  __shared__ double red[KRY_MAXM + 1][KRY_THREADS / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i <= KRY_MAXM; ++i) {
    if (i >= n) break;
    double a = acc[i].value();
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) red[i][warp] = a;
  }
  __syncthreads();
  if (threadIdx.x < n) {
    double a = 0.0;
    for (int k = 0; k < KRY_THREADS / 32; ++k) a += red[threadIdx.x][k];
    S->part[threadIdx.x * KRY_GRID + blockIdx.x] = a;
  }
}

// part[i][cta] = this CTA's share of w . v_i (i < n)
__global__ void __launch_bounds__(KRY_THREADS) k_kdot(const int32_t* __restrict__ tiles, int ntiles, int nx, int ny,
                                                      int pitch, const float* __restrict__ w, KryVecs V, int n,
                                                      KryScalars* __restrict__ S) {
  pdl_enter();
  Comp acc[KRY_MAXM + 1];
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    long p;
    if (!kcell(tiles, t, nx, ny, pitch, p)) continue;
    const float wv = w[p];
#pragma unroll
    for (int i = 0; i <= KRY_MAXM; ++i)
      if (i < n) acc[i].add(wv * V.v[i][p]);
  }
  kpartials(acc, n, S);
}

// one CTA adds the partial sums of n vectors in a fixed order, then:
//   mode 0 (Gram-Schmidt pass of column j): c[i] = s_i, H[i][j] += s_i;
//   mode 1 (new basis vector of column j):  H[j + 1][j] = sqrt(s_0), c[0] = 1 / that (0 if 0);
//   mode 2 (start of the step):              beta = sqrt(s_0), c[0] = 1 / beta (0 if 0)
__global__ void __launch_bounds__(KRY_THREADS) k_kreduce(int n, int mode, int j, int m, KryScalars* __restrict__ S) {
  pdl_enter();
  __shared__ double red[KRY_THREADS / 32];
  for (int i = 0; i < n; ++i) {
    double a = 0.0;
    for (int k = threadIdx.x; k < KRY_GRID; k += KRY_THREADS) a += S->part[i * KRY_GRID + k];
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int k = 0; k < KRY_THREADS / 32; ++k) s += red[k];
      if (mode == 0) {
        S->c[i] = s;
        S->H[j * (m + 1) + i] += s;
      } else {
        const double nrm = sqrt(fmax(s, 0.0));
        if (mode == 1) S->H[j * (m + 1) + j + 1] = nrm;
        else S->beta = nrm;
        S->c[0] = nrm > 0.0 ? 1.0 / nrm : 0.0;
      }
    }
    __syncthreads();
  }
}

// w -= sum_{i < n} c[i] v_i on the non-empty cells, then this CTA's share of the dot products
// of the new w with v_0 .. v_{n-1} (self = false) or with itself (self = true)
__global__ void __launch_bounds__(KRY_THREADS) k_ksubdot(const int32_t* __restrict__ tiles, int ntiles, int nx, int ny,
                                                         int pitch, const uint8_t* __restrict__ cls,
                                                         float* __restrict__ w, KryVecs V, int n, bool self,
                                                         KryScalars* __restrict__ S) {
  pdl_enter();
  float c[KRY_MAXM + 1];
#pragma unroll
  for (int i = 0; i <= KRY_MAXM; ++i) c[i] = i < n ? (float)S->c[i] : 0.f;
  Comp acc[KRY_MAXM + 1];
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    long p;
    if (!kcell(tiles, t, nx, ny, pitch, p) || cls[p] == 0) continue;
    float a = w[p];
    float v[KRY_MAXM + 1];
#pragma unroll
    for (int i = 0; i <= KRY_MAXM; ++i)
      if (i < n) {
        v[i] = V.v[i][p];
        a = fmaf(-c[i], v[i], a);
      }
    w[p] = a;
    if (self) {
      acc[0].add(a * a);
    } else {
#pragma unroll
      for (int i = 0; i <= KRY_MAXM; ++i)
        if (i < n) acc[i].add(a * v[i]);
    }
  }
  kpartials(acc, self ? 1 : n, S);
}

// out = c[0] x (out may be x) and, when r != nullptr, r = out too (the preconditioner's input)
__global__ void __launch_bounds__(KRY_THREADS) k_kscale(const int32_t* __restrict__ tiles, int ntiles, int nx, int ny,
                                                        int pitch, const uint8_t* __restrict__ cls, const float* x,
                                                        float* out, float* __restrict__ r,
                                                        const KryScalars* __restrict__ S) {
  pdl_enter();
  const float c0 = (float)S->c[0];
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    long p;
    if (!kcell(tiles, t, nx, ny, pitch, p) || cls[p] == 0) continue;
    const float v = c0 * x[p];
    out[p] = v;
    if (r) r[p] = v;
  }
}

// w = (h^2 L) z on the regular cells (FP32 stencil) and zj = z on every non-empty cell; the
// fitted rows of the irregular cells are applied by k_rows afterwards
template <bool CROSS>
__global__ void __launch_bounds__(KRY_THREADS) k_kapply(const int32_t* __restrict__ tiles, int nx, int ny, int pitch,
                                                        const uint8_t* __restrict__ cls, const float* __restrict__ z,
                                                        float* __restrict__ w, float* __restrict__ zj,
                                                        Stencil<float> St) {
  pdl_enter();
  const int i = tiles[2 * blockIdx.x] * TX + (threadIdx.x & 31);
  const int j = tiles[2 * blockIdx.x + 1] * TY + (threadIdx.x >> 5);
  if (i >= nx || j >= ny) return;
  const long p = (long)(j + 2) * pitch + (i + 2);
  const uint8_t c = cls[p];
  if (c == 0) return;
  zj[p] = z[p];
  if (c == 1) w[p] = stencil_apply<float, CROSS>(z, p, pitch, St);
}

// y = argmin || beta e_1 - H y ||_2 by Givens rotations (one thread; m <= KRY_MAXM).  A zero
// subdiagonal (the Krylov space became invariant) ends the basis there.
__global__ void k_klsq(int m, KryScalars* __restrict__ S) {
  pdl_enter();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double R[KRY_MAXM + 1][KRY_MAXM];
  double g[KRY_MAXM + 1];
  for (int jj = 0; jj < m; ++jj)
    for (int ii = 0; ii <= m; ++ii) R[ii][jj] = S->H[jj * (m + 1) + ii];
  for (int ii = 0; ii <= m; ++ii) g[ii] = 0.0;
  g[0] = S->beta;
  int k = m;
  for (int jj = 0; jj < m; ++jj) {
    const double a = R[jj][jj], b = R[jj + 1][jj];
    const double r = hypot(a, b);
    if (r == 0.0) {
      k = jj;
      break;
    }
    const double cs = a / r, sn = b / r;
    for (int q = jj; q < m; ++q) {
      const double x = R[jj][q], yv = R[jj + 1][q];
      R[jj][q] = cs * x + sn * yv;
      R[jj + 1][q] = -sn * x + cs * yv;
    }
    const double gx = g[jj], gy = g[jj + 1];
    g[jj] = cs * gx + sn * gy;
    g[jj + 1] = -sn * gx + cs * gy;
    if (b == 0.0) {        // invariant subspace: the columns after jj add nothing
      k = jj + 1;
      break;
    }
  }
  for (int q = m - 1; q >= 0; --q) {
    if (q >= k) {
      S->y[q] = 0.0;
      continue;
    }
    double a = g[q];
    for (int t = q + 1; t < k; ++t) a -= R[q][t] * S->y[t];
    S->y[q] = a / R[q][q];
  }
}

// u_hat += sum_{j < n} y_j z_j on the non-empty cells (the sum in FP32, the update in FP64)
__global__ void __launch_bounds__(KRY_THREADS) k_kupdate(const int32_t* __restrict__ tiles, int ntiles, int nx, int ny,
                                                         int pitch, const uint8_t* __restrict__ cls, KryVecs Z, int n,
                                                         const KryScalars* __restrict__ S, double* __restrict__ u) {
  pdl_enter();
  float y[KRY_MAXM];
#pragma unroll
  for (int k = 0; k < KRY_MAXM; ++k) y[k] = k < n ? (float)S->y[k] : 0.f;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    long p;
    if (!kcell(tiles, t, nx, ny, pitch, p) || cls[p] == 0) continue;
    float a = 0.f;
#pragma unroll
    for (int k = 0; k < KRY_MAXM; ++k)
      if (k < n) a = fmaf(y[k], Z.v[k][p], a);
    u[p] += (double)a;
  }
}

}  // namespace dev
}  // namespace ccm
