// The FP64 part of one outer iteration of the mixed-precision solve (eq.
// PoissonResidualForm): u_hat += e on the non-empty cells, then t = r_hat - (h^2 L) u_hat in
// FP64, the FP32 image of t as the next right-hand side of the FP32 V-cycles, and max |t|.
//
// The regular stencil (Sec. 3.2) is the sum of eq. stdLap along x and along y and the
// iterated eq. stdGrad for the mixed term, so its 25 weights factor as
//   w[dj][di] = a lap[di] / 12 [dj = 0] + c lap[dj] / 12 [di = 0] + (b grad[dj] / 12)(grad[di] / 12)
// with lap = (-1, 16, -30, 16, -1), grad = (1, -8, 0, 8, -1).  The kernel forms the x
// derivative grad_x u of every row of the staged tile once (4 FMA per cell) and combines
// four of them per cell, so a regular cell costs 4 + 4 + 9 FMA instead of 25 (FP64 issue is
// the bound of this kernel on GB300; the max-norm runs on the integer pipe).  The evaluation order differs from the 25-tap sum, so
// the result agrees with it to rounding, not bit for bit.
#pragma once

#include "kernels.cuh"

namespace ccm {
namespace dev {

struct SepStencil {
  double lx[5];    // a lap / 12 along x
  double ly[5];    // c lap / 12 along y
  double gx[5];    // grad / 12 along x
  double gy[5];    // b grad / 12 along y
  double cc;       // the centre weight (a + c) lap[2] / 12
};

// |t| as the bit pattern of a non-negative double, NaN mapped to +Inf: non-negative doubles
// order like their patterns, so the max-norm runs on the integer pipe
__device__ __forceinline__ unsigned long long abs_bits(double t) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(t) & 0x7fffffffffffffffULL;
  return b > 0x7ff0000000000000ULL ? 0x7ff0000000000000ULL : b;
}

// dynamic shared memory of k_resid64 (offsets are multiples of 128 bytes)
struct Resid64Smem {
  static constexpr uint32_t u_bytes = HY * HX * 8, r_bytes = JY * HX * 8, c_bytes = HY * CLX;
  static constexpr uint32_t rt_off = u_bytes;                          // 19584
  static constexpr uint32_t ct_off = rt_off + r_bytes;                 // 36992
  static constexpr uint32_t dx_off = ct_off + ((c_bytes + 127) / 128) * 128;
  static constexpr uint32_t tx = u_bytes + r_bytes + c_bytes;
  static constexpr uint32_t bytes(bool cross) { return cross ? dx_off + HY * JX * 8 : dx_off; }
};

// regular cells of one 64 x 32 tile: u_hat (68 x 36 halo), r_hat (68 x 32) and the class
// bytes (80 x 36) by TMA; writes r32 and folds max |t| into *norm
template <bool CROSS>
__global__ void __launch_bounds__(256, 3) k_resid64(const __grid_constant__ CUtensorMap tu,
                                                 const __grid_constant__ CUtensorMap tr,
                                                 const __grid_constant__ CUtensorMap tcls,
                                                 const int32_t* __restrict__ tiles, int nx, int pitch,
                                                 float* __restrict__ r32, unsigned long long* __restrict__ norm,
                                                 SepStencil S, int* __restrict__ err, long bs) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  double* ut = reinterpret_cast<double*>(smem_raw);                               // [HY][HX]
  double* rt = reinterpret_cast<double*>(smem_raw + Resid64Smem::rt_off);         // [JY][HX]
  uint8_t* ct = smem_raw + Resid64Smem::ct_off;                                   // [HY][CLX]
  double* dx = reinterpret_cast<double*>(smem_raw + Resid64Smem::dx_off);         // [HY][JX]
  __shared__ __align__(8) uint64_t bar;
  // while the previous launch drains: the tile's origin, the copy barrier and the class
  // bytes (static), with the byte count of the whole copy
  const int cx0 = tiles[2 * blockIdx.x] * JX, cy0 = tiles[2 * blockIdx.x + 1] * JY;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_expect_tx(&bar, Resid64Smem::tx);
    tma_load_2d(smem_raw + Resid64Smem::ct_off, &tcls, &bar, cx0, cy0);
  }
  __syncthreads();
  pdl_enter();
  const int z = blockIdx.y;          // right-hand side of the batch
  r32 += (long)z * bs;
  norm += z;
  if (threadIdx.x == 0) {
    tma_load_3d(ut, &tu, &bar, cx0, cy0, z);
    tma_load_3d(rt, &tr, &bar, cx0, cy0 + 2, z);
  }
  const bool ok = __syncthreads_and(tile_wait(&bar, err));
  if (!ok) return;
  if (CROSS) {
    for (int idx = threadIdx.x; idx < HY * JX; idx += blockDim.x) {
      const int y = idx >> 6, x = idx & 63;
      const double* row = ut + y * HX + x + 2;
      dx[idx] = S.gx[0] * row[-2] + S.gx[1] * row[-1] + S.gx[3] * row[1] + S.gx[4] * row[2];
    }
    __syncthreads();
  }
  // the 8 cells of a thread are independent: their arithmetic runs unconditionally, one FMA
  // chain each, so that the chains interleave; only the store depends on the class
  const int x = threadIdx.x & 63, y0 = (threadIdx.x >> 6) * 8;
  const int i = cx0 + x;
  unsigned long long m = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int y = y0 + k;                 // own row; staged row y + 2
    const double* c = ut + (y + 2) * HX + x + 2;
    double acc = S.cc * c[0];
    acc = fma(S.lx[0], c[-2], acc);
    acc = fma(S.lx[1], c[-1], acc);
    acc = fma(S.lx[3], c[1], acc);
    acc = fma(S.lx[4], c[2], acc);
    acc = fma(S.ly[0], c[-2 * HX], acc);
    acc = fma(S.ly[1], c[-HX], acc);
    acc = fma(S.ly[3], c[HX], acc);
    acc = fma(S.ly[4], c[2 * HX], acc);
    if (CROSS) {
      const double* d = dx + (y + 2) * JX + x;
      acc = fma(S.gy[0], d[-2 * JX], acc);
      acc = fma(S.gy[1], d[-JX], acc);
      acc = fma(S.gy[3], d[JX], acc);
      acc = fma(S.gy[4], d[2 * JX], acc);
    }
    const double t = rt[y * HX + x + 2] - acc;
    if (i < nx && ct[(y + 2) * CLX + x + 2] == 1) {
      r32[(long)(cy0 + y + 2) * pitch + (i + 2)] = (float)t;
      m = max(m, abs_bits(t));
    }
  }
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(norm, m);
}

// ---- the same residual in float-float arithmetic (pairs of FP32 words, about 48 bits).
// GB300 issues FP64 at 1/64 of the FP32 rate, so the FP64 kernel above is bound by its
// arithmetic.  Here the staged FP64 values are split into (hi, lo) FP32 pairs by integer
// operations (hi = the leading 24 significant bits, lo the next 24, both truncated), and the
// stencil runs in the integer-weight form of eq. stdLap and eq. stdGrad,
//   t = r_hat - [ a/12 Lap_x u + c/12 Lap_y u + b/144 Grad_y Grad_x u ],
//   Lap = 16 (u_-1 + u_+1) - (u_-2 + u_+2) - 30 u_0,  Grad = (u_-2 - u_+2) + 8 (u_+1 - u_-1),
// with every sum of leading words error-free (TwoSum) and the rounding errors, the low words
// and the errors of the products (FMA) carried in a second word.  The absolute error of t is
// about 2^-47 times the sum of the stencil's terms, 1e-13 relative to u here, against
// rounding at 2^-53 in FP64: good for relative residuals down to about 1e-11.

struct FFStencil {
  float ah, al;    // a / 12 as hi + lo
  float ch, cl;    // c / 12
  float bh, bl;    // b / 144
};

// hi + lo = x to 48 significant bits, by integer operations only; |x| below 2^-126 gives 0,
// Inf and NaN pass to hi (lo = 0)
__device__ __forceinline__ float2 ff_split(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned h32 = (unsigned)(b >> 32), l32 = (unsigned)b;
  const unsigned sign = h32 & 0x80000000u;
  const int e = (int)((h32 >> 20) & 0x7ffu);
  if (e == 0x7ff) return make_float2(__uint_as_float(sign | 0x7f800000u | (((h32 & 0xfffffu) | l32) ? 0x400000u : 0u)), 0.f);
  const int ef = e - 1023 + 127;
  if (ef <= 0) return make_float2(__uint_as_float(sign), 0.f);
  if (ef >= 255) return make_float2(__uint_as_float(sign | 0x7f800000u), 0.f);
  const unsigned m23 = ((h32 & 0xfffffu) << 3) | (l32 >> 29);
  const float hi = __uint_as_float(sign | ((unsigned)ef << 23) | m23);
  const unsigned rem = l32 & 0x1fffffffu;             // the 29 bits below hi, weight 2^(e - 1075)
  if (rem == 0u) return make_float2(hi, 0.f);
  const int lz = __clz(rem);                           // >= 3
  const int el = (31 - lz) + (e - 1075) + 127;
  if (el <= 0) return make_float2(hi, 0.f);
  const unsigned ml = ((rem << lz) >> 8) & 0x7fffffu;
  return make_float2(hi, __uint_as_float(sign | ((unsigned)el << 23) | ml));
}

struct FF {
  float s, e;      // value s + e
};

__device__ __forceinline__ FF ff(float2 v) { return FF{v.x, v.y}; }

// x + y, the sum of the leading words error-free (TwoSum)
__device__ __forceinline__ FF ff_add(FF x, FF y) {
  FF r;
  r.s = x.s + y.s;
  const float bb = r.s - x.s;
  r.e = ((x.s - (r.s - bb)) + (y.s - bb)) + (x.e + y.e);
  return r;
}
__device__ __forceinline__ FF ff_sub(FF x, FF y) { return ff_add(x, FF{-y.s, -y.e}); }
// p x for a power of two p (exact)
__device__ __forceinline__ FF ff_pow2(FF x, float p) { return FF{x.s * p, x.e * p}; }
// w x, the product of the leading word error-free (FMA)
__device__ __forceinline__ FF ff_mul(FF x, float w) {
  FF r;
  r.s = x.s * w;
  r.e = fmaf(x.e, w, fmaf(x.s, w, -r.s));
  return r;
}
// (ch + cl) x
__device__ __forceinline__ FF ff_mulc(FF x, float ch, float cl) {
  FF r;
  r.s = x.s * ch;
  r.e = fmaf(x.e, ch, fmaf(x.s, cl, fmaf(x.s, ch, -r.s)));
  return r;
}
// eq. stdLap's integer weights along a line: 16 (m1 + p1) - (m2 + p2) - 30 c
__device__ __forceinline__ FF ff_lap(FF m2, FF m1, FF c, FF p1, FF p2) {
  return ff_sub(ff_sub(ff_pow2(ff_add(m1, p1), 16.f), ff_add(m2, p2)), ff_mul(c, 30.f));
}
// eq. stdGrad's integer weights along a line: (m2 - p2) + 8 (p1 - m1)
__device__ __forceinline__ FF ff_grad(FF m2, FF m1, FF p1, FF p2) {
  return ff_add(ff_sub(m2, p2), ff_pow2(ff_sub(p1, m1), 8.f));
}

template <bool CROSS>
__global__ void __launch_bounds__(256, 3) k_resid_ff(const __grid_constant__ CUtensorMap tu,
                                                  const __grid_constant__ CUtensorMap tr,
                                                  const __grid_constant__ CUtensorMap tcls,
                                                  const int32_t* __restrict__ tiles, int nx, int pitch,
                                                  float* __restrict__ r32, unsigned long long* __restrict__ norm,
                                                  FFStencil S, int* __restrict__ err, long bs) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  double* ut = reinterpret_cast<double*>(smem_raw);                               // [HY][HX]
  const double* rt = reinterpret_cast<const double*>(smem_raw + Resid64Smem::rt_off);   // [JY][HX]
  const uint8_t* ct = smem_raw + Resid64Smem::ct_off;                             // [HY][CLX]
  float2* dx = reinterpret_cast<float2*>(smem_raw + Resid64Smem::dx_off);         // [HY][JX]
  __shared__ __align__(8) uint64_t bar;
  // while the previous launch drains: the tile's origin, the copy barrier and the class
  // bytes (static), with the byte count of the whole copy
  const int cx0 = tiles[2 * blockIdx.x] * JX, cy0 = tiles[2 * blockIdx.x + 1] * JY;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_expect_tx(&bar, Resid64Smem::tx);
    tma_load_2d(smem_raw + Resid64Smem::ct_off, &tcls, &bar, cx0, cy0);
  }
  __syncthreads();
  pdl_enter();
  const int z = blockIdx.y;          // right-hand side of the batch
  r32 += (long)z * bs;
  norm += z;
  if (threadIdx.x == 0) {
    tma_load_3d(ut, &tu, &bar, cx0, cy0, z);
    tma_load_3d(smem_raw + Resid64Smem::rt_off, &tr, &bar, cx0, cy0 + 2, z);
  }
  const bool ok = __syncthreads_and(tile_wait(&bar, err));
  if (!ok) return;
  // every staged value of u becomes its (hi, lo) pair in place
  float2* uf = reinterpret_cast<float2*>(ut);
  for (int idx = threadIdx.x; idx < HY * HX; idx += blockDim.x) {
    const float2 v = ff_split(ut[idx]);
    uf[idx] = v;
  }
  __syncthreads();
  if (CROSS) {
    for (int idx = threadIdx.x; idx < HY * JX; idx += blockDim.x) {
      const int y = idx >> 6, x = idx & 63;
      const float2* row = uf + y * HX + x + 2;
      const FF d = ff_grad(ff(row[-2]), ff(row[-1]), ff(row[1]), ff(row[2]));
      dx[idx] = make_float2(d.s, d.e);
    }
    __syncthreads();
  }
  const int x = threadIdx.x & 63, y0 = (threadIdx.x >> 6) * 8;
  const int i = cx0 + x;
  unsigned m = 0;
#pragma unroll 2
  for (int k = 0; k < 8; ++k) {
    const int y = y0 + k;                 // own row; staged row y + 2
    const float2* c = uf + (y + 2) * HX + x + 2;
    const FF c0 = ff(c[0]);
    const FF lx = ff_lap(ff(c[-2]), ff(c[-1]), c0, ff(c[1]), ff(c[2]));
    const FF ly = ff_lap(ff(c[-2 * HX]), ff(c[-HX]), c0, ff(c[HX]), ff(c[2 * HX]));
    FF lu = ff_add(ff_mulc(lx, S.ah, S.al), ff_mulc(ly, S.ch, S.cl));
    if (CROSS) {
      const float2* d = dx + (y + 2) * JX + x;
      lu = ff_add(lu, ff_mulc(ff_grad(ff(d[-2 * JX]), ff(d[-JX]), ff(d[JX]), ff(d[2 * JX])), S.bh, S.bl));
    }
    const FF t = ff_sub(ff(ff_split(rt[y * HX + x + 2])), lu);
    const float tf = t.s + t.e;
    if (i < nx && ct[(y + 2) * CLX + x + 2] == 1) {
      r32[(long)(cy0 + y + 2) * pitch + (i + 2)] = tf;
      unsigned b = __float_as_uint(tf) & 0x7fffffffu;
      m = max(m, b > 0x7f800000u ? 0x7f800000u : b);
    }
  }
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(norm, abs_bits((double)__uint_as_float(m)));
}

// fitted rows of the irregular cells: t = r_hat - sum_k beta_k u_hat(col_k); r32 and max |t|
__global__ void __launch_bounds__(128, 8) k_rows_r32(int n2, int W, const int32_t* __restrict__ cell, const int32_t* __restrict__ col,
                           const double* __restrict__ val, const double* __restrict__ u,
                           const double* __restrict__ r, float* __restrict__ r32,
                           unsigned long long* __restrict__ norm, long bs) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  // the row's cell, columns and coefficients (static) while the previous launch drains
  const int q = row < n2 ? cell[row] : 0;
  if (row < n2)
    for (int k = 0; k < W; ++k) {
      prefetch_l1(col + (long)k * n2 + row);
      prefetch_l1(val + (long)k * n2 + row);
    }
  pdl_enter();
  u += blockIdx.y * bs;       // right-hand side blockIdx.y of the batch
  r += blockIdx.y * bs;
  r32 += blockIdx.y * bs;
  norm += blockIdx.y;
  unsigned long long m = 0;
  if (row < n2) {
    double acc = 0.0;
#pragma unroll 15
    for (int k = 0; k < W; ++k) acc += val[(long)k * n2 + row] * u[col[(long)k * n2 + row]];
    const double t = r[q] - acc;
    r32[q] = (float)t;
    m = abs_bits(t);
  }
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(norm, m);
}

// u_hat += e on the non-empty cells of the 32 x 8 tiles that hold one
__global__ void k_axpy_tiles(const int32_t* __restrict__ tiles, const uint8_t* __restrict__ cls, int nx, int ny,
                             int pitch, const float* __restrict__ e, double* __restrict__ u, long bs) {
  // the cell and its class (static) while the previous launch drains
  const int i = tiles[2 * blockIdx.x] * TX + threadIdx.x;
  const int j = tiles[2 * blockIdx.x + 1] * TY + threadIdx.y;
  const long p = (long)(j + 2) * pitch + (i + 2);
  const bool on = i < nx && j < ny && cls[p] != 0;
  pdl_enter();
  e += blockIdx.y * bs;       // right-hand side blockIdx.y of the batch
  u += blockIdx.y * bs;
  if (on) u[p] += (double)e[p];
}

}  // namespace dev
}  // namespace ccm
