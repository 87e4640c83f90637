// Device kernels of the V-cycle (Sec. 4) on the padded level layout.
//
// Every level is a padded [rows][pitch] array (2-cell zero ring), cell classes in `cls`
// (0 empty or ring, 1 regular, 2 irregular).  All arithmetic is on the h^2-scaled system
// (h^2 L) u = h^2 r, so the regular stencil is the same 25 constants on every level.
// Regular cells run on 32 x 8 tiles (one thread per cell, empty tiles skipped); the fitted
// rows of irregular cells are ELL with 15 slots, one thread per row.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ccm {
namespace dev {

constexpr int TX = 32, TY = 8;

template <typename T>
struct Stencil {
  T w[25];        // [dj + 2][di + 2]
  T omega_d;      // omega / w[2][2] (SMO-1 weight over the diagonal)
};

// (h^2 L u) at a regular cell: 9-point cross (b = 0) or the full 5 x 5 box
template <typename T, bool CROSS>
__device__ __forceinline__ T stencil_apply(const T* __restrict__ u, long p, int pitch, const Stencil<T>& S) {
  T acc = S.w[12] * u[p];
  acc += S.w[10] * u[p - 2] + S.w[11] * u[p - 1] + S.w[13] * u[p + 1] + S.w[14] * u[p + 2];
  acc += S.w[2] * u[p - 2 * pitch] + S.w[7] * u[p - pitch] + S.w[17] * u[p + pitch] + S.w[22] * u[p + 2 * pitch];
  if (CROSS) {
#pragma unroll
    for (int dj = -2; dj <= 2; ++dj) {
      if (dj == 0) continue;
#pragma unroll
      for (int di = -2; di <= 2; ++di) {
        if (di == 0) continue;
        acc += S.w[(dj + 2) * 5 + di + 2] * u[p + (long)dj * pitch + di];
      }
    }
  }
  return acc;
}

__device__ __forceinline__ bool tile_cell(const int32_t* __restrict__ tiles, int nx, int ny, int pitch, int& i,
                                          int& j, long& p) {
  i = tiles[2 * blockIdx.x] * TX + threadIdx.x;
  j = tiles[2 * blockIdx.x + 1] * TY + threadIdx.y;
  p = (long)(j + 2) * pitch + (i + 2);
  return i < nx && j < ny;
}

// SMO-1 (Sec. 4.1): u_out = u_in + omega D^-1 (r - L u_in) on regular cells, copy elsewhere
template <typename T, bool CROSS>
__global__ void k_jacobi(const int32_t* __restrict__ tiles, const uint8_t* __restrict__ cls, int nx, int ny,
                         int pitch, const T* __restrict__ u_in, T* __restrict__ u_out, const T* __restrict__ r,
                         Stencil<T> S) {
  int i, j;
  long p;
  if (!tile_cell(tiles, nx, ny, pitch, i, j, p)) return;
  uint8_t c = cls[p];
  if (c == 1) {
    T Lu = stencil_apply<T, CROSS>(u_in, p, pitch, S);
    u_out[p] = u_in[p] + S.omega_d * (r[p] - Lu);
  } else if (c == 2) {
    u_out[p] = u_in[p];
  }
}

// out = r - L u on regular cells (sign = +1) or out = L u (sign = 0)
template <typename T, bool CROSS, bool RESID>
__global__ void k_regular(const int32_t* __restrict__ tiles, const uint8_t* __restrict__ cls, int nx, int ny,
                          int pitch, const T* __restrict__ u, const T* __restrict__ r, T* __restrict__ out,
                          Stencil<T> S) {
  int i, j;
  long p;
  if (!tile_cell(tiles, nx, ny, pitch, i, j, p)) return;
  if (cls[p] != 1) return;
  T Lu = stencil_apply<T, CROSS>(u, p, pitch, S);
  out[p] = RESID ? r[p] - Lu : Lu;
}

// fitted rows: res = r[cell] - sum beta u[col]  (RESID) or res = sum beta u[col] + nb g[seg]
// written to out[row] (GRID = false) or out[cell] (GRID = true)
template <typename T, typename C, bool RESID, bool GRID>
__global__ void k_rows(int n2, const int32_t* __restrict__ cell, const int32_t* __restrict__ col,
                       const C* __restrict__ val, const T* __restrict__ u, const T* __restrict__ r,
                       T* __restrict__ out, const double* __restrict__ nb, const int32_t* __restrict__ seg,
                       const double* __restrict__ g) {
  int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n2) return;
  T acc = 0;
#pragma unroll
  for (int k = 0; k < 15; ++k) acc += (T)val[(long)k * n2 + row] * u[col[(long)k * n2 + row]];
  T res;
  if (RESID) {
    res = r[cell[row]] - acc;
  } else {
    res = acc;
    if (g != nullptr && seg[row] >= 0) res += (T)(nb[row] * g[seg[row]]);
  }
  if (GRID) out[cell[row]] = res;
  else out[row] = res;
}

// SMO-2 (Sec. 4.1) as one pass of overlapping block solves: for every block, the core
// unknowns get inv(L22[ext, ext])[core, :] applied to the residuals of the extended block.
// Grid (block, chunk of 32 core rows); the 4 warps of a CTA split the extended range.
template <typename T>
__global__ void k_block_solve(const int32_t* __restrict__ order, const int32_t* __restrict__ blk,
                              const int64_t* __restrict__ blk_off, const T* __restrict__ inv,
                              const T* __restrict__ res2, const int32_t* __restrict__ cell, T* __restrict__ u) {
  extern __shared__ unsigned char smem_raw[];
  T* s = reinterpret_cast<T*>(smem_raw);
  __shared__ T part[4][32];
  const int b = blockIdx.x;
  const int cs = blk[4 * b], ce = blk[4 * b + 1], es = blk[4 * b + 2], ee = blk[4 * b + 3];
  const int ne = ee - es, nc = ce - cs;
  const int c0 = blockIdx.y * 32;
  if (c0 >= nc) return;
  for (int e = threadIdx.x; e < ne; e += blockDim.x) s[e] = res2[order[es + e]];
  __syncthreads();
  const T* A = inv + blk_off[b];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = c0 + lane;
  T acc = 0;
  if (c < nc)
    for (int e = warp; e < ne; e += 4) acc += A[(long)e * nc + c] * s[e];
  part[warp][lane] = acc;
  __syncthreads();
  if (warp == 0 && c < nc) {
    T tot = part[0][lane] + part[1][lane] + part[2][lane] + part[3][lane];
    u[cell[order[cs + c]]] += tot;
  }
}

// SMO-1 with the prolongation fused in (first post-smoothing sweep after Alg. 2's
// "Prolong the correction"): v = u + P uc on regular cells, then u_out = v + omega D^-1 (r - L v)
// on regular cells.  Irregular cells are left to the SMO-2 kernel that follows.
template <typename T, bool CROSS, bool PROLONG>
__global__ void k_jacobi2(const int32_t* __restrict__ tiles, const uint8_t* __restrict__ cls, int nx, int ny,
                          int pitch, int pitchc, const T* __restrict__ u_in, const T* __restrict__ uc,
                          T* __restrict__ u_out, const T* __restrict__ r, Stencil<T> S) {
  int i, j;
  long p;
  if (!tile_cell(tiles, nx, ny, pitch, i, j, p)) return;
  if (cls[p] != 1) return;
  T acc = 0;
  T vp = 0;
#pragma unroll
  for (int dj = -2; dj <= 2; ++dj)
#pragma unroll
    for (int di = -2; di <= 2; ++di) {
      if (!CROSS && dj != 0 && di != 0) continue;
      long q = p + (long)dj * pitch + di;
      T v = u_in[q];
      if (PROLONG && cls[q] == 1) v += uc[(long)((j + dj) / 2 + 2) * pitchc + ((i + di) / 2 + 2)];
      acc += S.w[(dj + 2) * 5 + di + 2] * v;
      if (dj == 0 && di == 0) vp = v;
    }
  u_out[p] = vp + S.omega_d * (r[p] - acc);
}

// SMO-2 fused with the residual of the fitted rows: the residual of row e uses the new
// regular values (u_new, written by SMO-1) and the old irregular values (u_old); the core
// rows of the block then get u_new = u_old + inv(L22[ext, ext])[core, :] res[ext].  Every
// irregular cell is the core of exactly one block, and no kernel writes what it reads.
template <typename T>
__global__ void k_block_fused(const int32_t* __restrict__ order, const int32_t* __restrict__ blk,
                              const int64_t* __restrict__ blk_off, const T* __restrict__ inv,
                              int n2, const int32_t* __restrict__ cell, const int32_t* __restrict__ col,
                              const T* __restrict__ val, const uint8_t* __restrict__ cls,
                              const T* __restrict__ r, const T* __restrict__ u_old, T* __restrict__ u_new) {
  extern __shared__ unsigned char smem_raw[];
  T* s = reinterpret_cast<T*>(smem_raw);
  __shared__ T part[4][32];
  const int b = blockIdx.x;
  const int cs = blk[4 * b], ce = blk[4 * b + 1], es = blk[4 * b + 2], ee = blk[4 * b + 3];
  const int ne = ee - es, nc = ce - cs;
  const int c0 = blockIdx.y * 32;
  if (c0 >= nc) return;
  for (int e = threadIdx.x; e < ne; e += blockDim.x) {
    int row = order[es + e];
    T acc = 0;
#pragma unroll
    for (int k = 0; k < 15; ++k) {
      int q = col[(long)k * n2 + row];
      T v = cls[q] == 1 ? u_new[q] : u_old[q];
      acc += val[(long)k * n2 + row] * v;
    }
    s[e] = r[cell[row]] - acc;
  }
  __syncthreads();
  const T* A = inv + blk_off[b];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = c0 + lane;
  T acc = 0;
  if (c < nc)
    for (int e = warp; e < ne; e += 4) acc += A[(long)e * nc + c] * s[e];
  part[warp][lane] = acc;
  __syncthreads();
  if (warp == 0 && c < nc) {
    long q = cell[order[cs + c]];
    u_new[q] = u_old[q] + part[0][lane] + part[1][lane] + part[2][lane] + part[3][lane];
  }
}

// residual + restriction + zeroing of the coarse iterate (Alg. 2 "compute the coarse
// residual by restriction" and "u^(m+1) = 0"): regular children's residuals are computed
// here, irregular children's are read from t (written by k_rows).
template <typename T, bool CROSS>
__global__ void k_restrict_fused(int nxc, int nyc, int pitchc, int pitchf, const uint8_t* __restrict__ clsc,
                                 const uint8_t* __restrict__ clsf, const T* __restrict__ volf,
                                 const T* __restrict__ u, const T* __restrict__ r, const T* __restrict__ t,
                                 T* __restrict__ rc, T* __restrict__ uc, Stencil<T> S) {
  int I = blockIdx.x * blockDim.x + threadIdx.x;
  int J = blockIdx.y * blockDim.y + threadIdx.y;
  if (I >= nxc || J >= nyc) return;
  long pc = (long)(J + 2) * pitchc + (I + 2);
  if (clsc[pc] == 0) return;
  long f0 = (long)(2 * J + 2) * pitchf + (2 * I + 2);
  T s = 0, sv = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    long q = f0 + (k >> 1) * (long)pitchf + (k & 1);
    uint8_t c = clsf[q];
    if (c == 0) continue;
    T res = c == 1 ? r[q] - stencil_apply<T, CROSS>(u, q, pitchf, S) : t[q];
    T v = volf[q];
    s += v * res;
    sv += v;
  }
  rc[pc] = sv > (T)0 ? (T)4 * s / sv : (T)0;
  uc[pc] = (T)0;
}

// residual restriction (Sec. 4.1), h^2-scaled: rc = 4 sum(vol t) / sum(vol) over the children
template <typename T>
__global__ void k_restrict(int nxc, int nyc, int pitchc, int pitchf, const uint8_t* __restrict__ clsc,
                           const T* __restrict__ volf, const T* __restrict__ t, T* __restrict__ rc) {
  int I = blockIdx.x * blockDim.x + threadIdx.x;
  int J = blockIdx.y * blockDim.y + threadIdx.y;
  if (I >= nxc || J >= nyc) return;
  long pc = (long)(J + 2) * pitchc + (I + 2);
  if (clsc[pc] == 0) return;
  long f0 = (long)(2 * J + 2) * pitchf + (2 * I + 2);
  T v0 = volf[f0], v1 = volf[f0 + 1], v2 = volf[f0 + pitchf], v3 = volf[f0 + pitchf + 1];
  T s = v0 * t[f0] + v1 * t[f0 + 1] + v2 * t[f0 + pitchf] + v3 * t[f0 + pitchf + 1];
  T sv = v0 + v1 + v2 + v3;
  rc[pc] = sv > (T)0 ? (T)4 * s / sv : (T)0;
}

// prolongation (Sec. 4.1): u += uc[parent] on fine regular cells
template <typename T>
__global__ void k_prolong(const int32_t* __restrict__ tiles, const uint8_t* __restrict__ cls, int nx, int ny,
                          int pitch, int pitchc, const T* __restrict__ uc, T* __restrict__ u) {
  int i, j;
  long p;
  if (!tile_cell(tiles, nx, ny, pitch, i, j, p)) return;
  if (cls[p] != 1) return;
  u[p] += uc[(long)(j / 2 + 2) * pitchc + (i / 2 + 2)];
}

// bottom solve: u[cell_k] = sum_c inv[c][k] r[cell_c]
template <typename T>
__global__ void k_bottom(int n, const int32_t* __restrict__ cell, const T* __restrict__ inv,
                         const T* __restrict__ r, T* __restrict__ u) {
  extern __shared__ unsigned char smem_raw[];
  T* s = reinterpret_cast<T*>(smem_raw);
  for (int c = threadIdx.x; c < n; c += blockDim.x) s[c] = r[cell[c]];
  __syncthreads();
  // each block computes a slice of rows, warps split the columns
  const int rows_per_block = 32;
  const int k = blockIdx.x * rows_per_block + (threadIdx.x & 31);
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T acc = 0;
  if (k < n)
    for (int c = warp; c < n; c += nw) acc += inv[(long)c * n + k] * s[c];
  __syncthreads();
  T* part = s;   // reuse: [nw][32]
  part[warp * 32 + (threadIdx.x & 31)] = acc;
  __syncthreads();
  if (warp == 0 && k < n) {
    T tot = 0;
    for (int w = 0; w < nw; ++w) tot += part[w * 32 + threadIdx.x];
    u[cell[k]] = tot;
  }
}

// ---- conversions and reductions on the padded layout

// padded <- user layout (non-empty cells only), scaled
template <typename TD, typename TS>
__global__ void k_pack(int nx, int ny, int pitch, const uint8_t* __restrict__ cls, const TS* __restrict__ src,
                       TD* __restrict__ dst, double scale) {
  int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= nx) return;
  long p = (long)(j + 2) * pitch + (i + 2);
  if (cls[p] != 0) dst[p] = (TD)(scale * (double)src[(long)j * nx + i]);
}

// user layout <- padded (0 for empty cells), scaled
template <typename TS>
__global__ void k_unpack(int nx, int ny, int pitch, const uint8_t* __restrict__ cls, const TS* __restrict__ src,
                         double* __restrict__ dst, double scale) {
  int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= nx) return;
  long p = (long)(j + 2) * pitch + (i + 2);
  dst[(long)j * nx + i] = cls[p] != 0 ? scale * (double)src[p] : 0.0;
}

// r_hat -= nb g on the rows that own a boundary segment
__global__ void k_sub_boundary(int n2, const int32_t* __restrict__ cell, const double* __restrict__ nb,
                               const int32_t* __restrict__ seg, const double* __restrict__ g, double* __restrict__ r) {
  int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n2 || seg[row] < 0) return;
  r[cell[row]] -= nb[row] * g[seg[row]];
}

// max |x| over the non-empty cells (non-negative doubles order like their bit patterns)
template <typename T>
__global__ void k_absmax(long n, const uint8_t* __restrict__ cls, const T* __restrict__ x,
                         unsigned long long* __restrict__ out) {
  double m = 0.0;
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < n; p += (long)gridDim.x * blockDim.x)
    if (cls[p] != 0) {
      double v = fabs((double)x[p]);
      if (!(v <= 1.7976931348623157e308)) v = __longlong_as_double(0x7ff0000000000000ULL);   // NaN -> Inf
      m = fmax(m, v);
    }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// u64 += e on non-empty cells;  r32 = (float) r64
template <typename TE>
__global__ void k_axpy(long n, const uint8_t* __restrict__ cls, const TE* __restrict__ e, double* __restrict__ u) {
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < n; p += (long)gridDim.x * blockDim.x)
    if (cls[p] != 0) u[p] += (double)e[p];
}
__global__ void k_to_float(long n, const double* __restrict__ a, float* __restrict__ b) {
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < n; p += (long)gridDim.x * blockDim.x)
    b[p] = (float)a[p];
}

// transposed operator, scatter-free: out[c] = sum_d w_d v[c + d] [c + d regular]
// (the regular stencil is point-symmetric) for every non-empty c ...
template <bool CROSS>
__global__ void k_regular_T(const int32_t* __restrict__ tiles, const uint8_t* __restrict__ cls, int nx, int ny,
                            int pitch, const double* __restrict__ v, double* __restrict__ out, Stencil<double> S) {
  int i, j;
  long p;
  if (!tile_cell(tiles, nx, ny, pitch, i, j, p)) return;
  if (cls[p] == 0) return;
  double acc = 0;
#pragma unroll
  for (int dj = -2; dj <= 2; ++dj)
#pragma unroll
    for (int di = -2; di <= 2; ++di) {
      double w = S.w[(dj + 2) * 5 + di + 2];
      if (!CROSS && dj != 0 && di != 0) continue;
      long q = p + (long)dj * pitch + di;
      if (cls[q] == 1) acc += w * v[q];
    }
  out[p] = acc;
}
// ... plus the fitted rows through the transposed CSR (one thread per column cell)
__global__ void k_rows_T(int ncol, const int32_t* __restrict__ ptr, const int32_t* __restrict__ ccell,
                         const int32_t* __restrict__ row, const double* __restrict__ val,
                         const int32_t* __restrict__ rcell, const double* __restrict__ v, double* __restrict__ out) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= ncol) return;
  double acc = 0;
  for (int e = ptr[k]; e < ptr[k + 1]; ++e) acc += val[e] * v[rcell[row[e]]];
  out[ccell[k]] += acc;
}
// N^T v: one entry per segment (each segment belongs to exactly one fitted row)
__global__ void k_bnd_T(int n2, const int32_t* __restrict__ cell, const double* __restrict__ nb,
                        const int32_t* __restrict__ seg, const double* __restrict__ v, double* __restrict__ og,
                        double scale) {
  int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n2 || seg[row] < 0) return;
  og[seg[row]] = scale * nb[row] * v[cell[row]];
}

}  // namespace dev
}  // namespace ccm
