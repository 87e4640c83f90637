// Device kernels of the V-cycle (Sec. 4) on the padded level layout.
//
// Every level is a padded [rows][pitch] array (2-cell zero ring), cell classes in `cls`
// (0 empty or ring, 1 regular, 2 irregular).  All arithmetic is on the h^2-scaled system
// (h^2 L) u = h^2 r, so the regular stencil is the same 25 constants on every level.
// Regular cells run on 32 x 8 tiles (one thread per cell, empty tiles skipped); the fitted
// rows of irregular cells are ELL with 15 slots, one thread per row.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace ccm {
namespace dev {

constexpr int TX = 32, TY = 8;

// Programmatic dependent launch: a kernel launched with programmatic stream serialization
// may start while the preceding kernel of its stream drains.  Every kernel of the solve path
// first waits for that kernel (and sees its writes) before it touches global memory, then
// lets the next kernel's CTAs be scheduled.  Without the launch attribute both are no-ops.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// hint: bring the line holding p into this SM's L1.  Kernels use it before pdl_enter() on
// static data (level structure, operator coefficients, tile lists), which no kernel of the
// solve writes, so that their first dependent loads after the wait hit L1
__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

template <typename T>
struct Stencil {
  T w[25];        // [dj + 2][di + 2]
  T omega_d;      // omega / w[2][2] (SMO-1 weight over the diagonal)
  // the same stencil factored: w[dj][di] = lx[di] [dj = 0] + ly[dj] [di = 0] + gy[dj] gx[di]
  // (eq. stdLap along x and y, the product of two eq. stdGrad derivatives for the mixed term)
  T lx[5], ly[5], gx[5], gy[5], cc;   // cc = lx[2] + ly[2]
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
  pdl_enter();
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
__global__ void __launch_bounds__(128, 8) k_rows(int n2, int W, const int32_t* __restrict__ cell, const int32_t* __restrict__ col,
                       const C* __restrict__ val, const T* __restrict__ u, const T* __restrict__ r,
                       T* __restrict__ out, const double* __restrict__ nb, const int32_t* __restrict__ seg,
                       const double* __restrict__ g) {
  pdl_enter();
  int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n2) return;
  T acc = 0;
#pragma unroll 15
  for (int k = 0; k < W; ++k) acc += (T)val[(long)k * n2 + row] * u[col[(long)k * n2 + row]];
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

// ---- TMA-staged SMO-1 for the large levels.
// A 64 x 32 tile of cells plus its 2-cell halo (68 x 36 values) is one 2-D TMA box: in the
// padded layout the halo of the tile at cells (64 a, 32 b) starts at padded column 64 a, a
// multiple of 16 bytes for every element size, and rows have no alignment rule.  Cells past
// the array edge read the zero fill.  256 threads: 64 columns x 4 groups of 8 rows, a 5 x 5
// register window slides down each column so that every cell costs 5 shared-memory loads.
constexpr int JX = 64, JY = 32, HX = JX + 4, HY = JY + 4;
constexpr long long TMA_WAIT_CYCLES = 4000000;   // ~2 ms at 2 GHz: bound on a tile wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// test for the completion of the phase with the given parity; the thread may stay suspended
// in the instruction for up to 100 us while the phase is pending (no issue slots spent)
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase), "r"(100000u)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// 3-D box (x, y, right-hand side z): the iterate and right-hand-side maps of a level cover
// all right-hand sides of a batch, one padded level array after the other
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// orders this thread's earlier shared-memory accesses before later async-proxy (TMA, bulk)
// writes into the same buffer
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// bounded wait for the tile (by the SM clock); false, and *err set, if the copy never landed
__device__ __forceinline__ bool tile_wait(uint64_t* bar, int* err) {
  const long long t0 = clock64();
  while (clock64() - t0 < TMA_WAIT_CYCLES)
    if (mbar_try_wait(bar, 0)) return true;
  if (threadIdx.x == 0) atomicExch(err, 1);
  const long long t1 = clock64();     // let the copy in flight finish before leaving
  while (clock64() - t1 < TMA_WAIT_CYCLES)
    if (mbar_try_wait(bar, 0)) break;
  return false;
}

template <typename T, bool CROSS>
__global__ void __launch_bounds__(256) k_jacobi_tma(const __grid_constant__ CUtensorMap tin,
                                                    const int32_t* __restrict__ tiles, const uint8_t* __restrict__ cls,
                                                    int nx, int ny, int pitch, const T* __restrict__ r,
                                                    T* __restrict__ u_out, Stencil<T> S, int* __restrict__ err) {
  __shared__ __align__(128) T tile[HY * HX];
  __shared__ __align__(8) uint64_t bar;
  const int cx0 = tiles[2 * blockIdx.x] * JX, cy0 = tiles[2 * blockIdx.x + 1] * JY;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_expect_tx(&bar, (uint32_t)(HX * HY * sizeof(T)));
    tma_load_3d(tile, &tin, &bar, cx0, cy0, 0);
  }
  // the class bytes and right-hand sides of this thread's 8 cells load while the tile lands
  const int x = threadIdx.x & 63, y0 = (threadIdx.x >> 6) * 8;
  const int i = cx0 + x;
  uint8_t cv[8];
  T rv[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int j = cy0 + y0 + k;
    const long p = (long)(j + 2) * pitch + (i + 2);
    const bool in = i < nx && j < ny;
    cv[k] = in ? cls[p] : (uint8_t)0;
    rv[k] = in ? r[p] : (T)0;
  }
  if (!tile_wait(&bar, err)) return;
  if (i >= nx) return;
  T w[5][5];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 5; ++b) w[a][b] = tile[(y0 + a) * HX + x + b];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
#pragma unroll
    for (int b = 0; b < 5; ++b) w[4][b] = tile[(y0 + k + 4) * HX + x + b];
    if (cv[k] == 1) {
      T acc = 0;
#pragma unroll
      for (int a = 0; a < 5; ++a)
#pragma unroll
        for (int b = 0; b < 5; ++b) {
          if (!CROSS && a != 2 && b != 2) continue;
          acc += S.w[a * 5 + b] * w[a][b];
        }
      const long p = (long)(cy0 + y0 + k + 2) * pitch + (i + 2);
      u_out[p] = w[2][2] + S.omega_d * (rv[k] - acc);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 5; ++b) w[a][b] = w[a + 1][b];
  }
}

// ---- one smoothing sweep in one launch (block-Jacobi form of SMO-1 + SMO-2).
// Both parts read only the old iterate and write only the new one: CTAs [0, ntiles) update
// the regular cells (SMO-1), CTAs [ntiles, ntiles + nblk * chunks) the irregular cells by the
// overlapping block solve (SMO-2 whose residual uses the old regular values).  The fixed
// point is the same as for SMO-1 followed by SMO-2.
template <typename T>
struct SweepArgs {
  const int32_t* tiles;      // TMA: 64 x 32 tiles, else 32 x 8 tiles
  int ntiles, nblk, chunks, rows_per_cta;
  const uint8_t* cls;
  int nx, ny, pitch, n2, W;
  const T* r;
  const T* u_old;
  T* u_new;
  Stencil<T> S;
  const int32_t* blk;
  const int64_t* blk_off;
  const T* inv;
  const int32_t* cell;
  const int32_t* col;
  const T* val;
  int* err;
  const int32_t* par;    // per ELL slot: padded parent (level m + 1) of a regular column, else -1
  const T* uc;           // coarse iterate: the sweep reads u + P uc (regular cells), or null
  long bs, bsc;          // batch strides (elements) of this level's and the coarse level's arrays
  // persistent sweep only: zero_u, the old iterate is 0 (it is not read); uhat (FP32 sweep of
  // level 0, or null), the FP64 solution to which every new value is added (u_hat += e as the
  // last sweep of an outer iteration writes e), same layout and batch stride
  int zero_u;
  double* uhat;
};

template <typename T>
__device__ __forceinline__ void block_part(const SweepArgs<T>& a, int bidx, T* s) {
  __shared__ T part[8][32];
  const int b = bidx / a.chunks, chunk = bidx % a.chunks;
  const int cs = a.blk[4 * b], ce = a.blk[4 * b + 1], es = a.blk[4 * b + 2], ee = a.blk[4 * b + 3];
  const int ne = ee - es, nc = ce - cs;
  const int c0 = chunk * a.rows_per_cta;
  if (c0 >= nc) return;
  for (int e = threadIdx.x; e < ne; e += blockDim.x) {
    const int row = es + e;
    T acc = 0;
#pragma unroll 15
    for (int k = 0; k < a.W; ++k) acc += a.val[(long)k * a.n2 + row] * a.u_old[a.col[(long)k * a.n2 + row]];
    s[e] = a.r[a.cell[row]] - acc;
  }
  __syncthreads();
  const T* A = a.inv + a.blk_off[b];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int cend = min(nc, c0 + a.rows_per_cta);
  for (int cb = c0; cb < cend; cb += 32) {
    const int c = cb + lane;
    T acc = 0;
    if (c < cend)
      for (int e = warp; e < ne; e += nw) acc += A[(long)e * nc + c] * s[e];
    part[warp][lane] = acc;
    __syncthreads();
    if (warp == 0 && c < cend) {
      T tot = 0;
      for (int w = 0; w < nw; ++w) tot += part[w][lane];
      const long q = a.cell[cs + c];
      a.u_new[q] = a.u_old[q] + tot;
    }
    __syncthreads();
  }
}

template <typename T, bool CROSS, bool TMA>
__global__ void __launch_bounds__(256) k_sweep(const __grid_constant__ CUtensorMap tin, SweepArgs<T> a) {
  pdl_enter();
  extern __shared__ unsigned char smem_raw[];
  a.u_old += (long)blockIdx.y * a.bs;      // right-hand side blockIdx.y of the batch
  a.u_new += (long)blockIdx.y * a.bs;
  a.r += (long)blockIdx.y * a.bs;
  if ((int)blockIdx.x >= a.ntiles) {
    block_part<T>(a, blockIdx.x - a.ntiles, reinterpret_cast<T*>(smem_raw));
    return;
  }
  const Stencil<T>& S = a.S;
  if (!TMA) {
    // 32 x 8 tile, one cell per thread
    const int i = a.tiles[2 * blockIdx.x] * TX + (threadIdx.x & 31);
    const int j = a.tiles[2 * blockIdx.x + 1] * TY + (threadIdx.x >> 5);
    if (i >= a.nx || j >= a.ny) return;
    const long p = (long)(j + 2) * a.pitch + (i + 2);
    if (a.cls[p] != 1) return;
    const T Lu = stencil_apply<T, CROSS>(a.u_old, p, a.pitch, S);
    a.u_new[p] = a.u_old[p] + S.omega_d * (a.r[p] - Lu);
    return;
  }
  __shared__ __align__(128) T tile[TMA ? HY * HX : 1];
  __shared__ __align__(8) uint64_t bar;
  const int cx0 = a.tiles[2 * blockIdx.x] * JX, cy0 = a.tiles[2 * blockIdx.x + 1] * JY;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_expect_tx(&bar, (uint32_t)(HX * HY * sizeof(T)));
    tma_load_3d(tile, &tin, &bar, cx0, cy0, 0);
  }
  const int x = threadIdx.x & 63, y0 = (threadIdx.x >> 6) * 8;
  const int i = cx0 + x;
  uint8_t cv[8];
  T rv[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int j = cy0 + y0 + k;
    const long p = (long)(j + 2) * a.pitch + (i + 2);
    const bool in = i < a.nx && j < a.ny;
    cv[k] = in ? a.cls[p] : (uint8_t)0;
    rv[k] = in ? a.r[p] : (T)0;
  }
  if (!tile_wait(&bar, a.err)) return;
  if (i >= a.nx) return;
  T w[5][5];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int b = 0; b < 5; ++b) w[q][b] = tile[(y0 + q) * HX + x + b];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
#pragma unroll
    for (int b = 0; b < 5; ++b) w[4][b] = tile[(y0 + k + 4) * HX + x + b];
    if (cv[k] == 1) {
      T acc = 0;
#pragma unroll
      for (int q = 0; q < 5; ++q)
#pragma unroll
        for (int b = 0; b < 5; ++b) {
          if (!CROSS && q != 2 && b != 2) continue;
          acc += S.w[q * 5 + b] * w[q][b];
        }
      const long p = (long)(cy0 + y0 + k + 2) * a.pitch + (i + 2);
      a.u_new[p] = w[2][2] + S.omega_d * (rv[k] - acc);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int b = 0; b < 5; ++b) w[q][b] = w[q + 1][b];
  }
}

// SMO-1 on one TMA-staged 64 x 32 tile (the regular cells; the SMO-2 blocks run in k_blocks
// beside it).  With PRO the sweep is the first post-smoothing sweep of Alg. 2 and reads
// u + P uc: the class bytes of the tile with its halo (80 x 36 box) and the coarse iterate
// under it (36 x 18 box, x origin cx0 / 2, a multiple of 32 elements) arrive with the same
// mbarrier, and the coarse correction is added to the regular cells of the staged tile
// before the stencil runs (Sec. 4.1: prolongation to regular cells only).
constexpr int CLX = 80, UCX = 36, UCY = HY / 2;

template <typename T, bool CROSS, bool PRO>
__global__ void __launch_bounds__(256) k_sweep_tma(const __grid_constant__ CUtensorMap tin,
                                                   const __grid_constant__ CUtensorMap tcls,
                                                   const __grid_constant__ CUtensorMap tuc, SweepArgs<T> a) {
  pdl_enter();
  __shared__ __align__(128) T tile[HY * HX];
  __shared__ __align__(128) uint8_t ctile[PRO ? HY * CLX : 16];
  __shared__ __align__(128) T uct[PRO ? UCY * UCX : 2];
  __shared__ __align__(8) uint64_t bar;
  const int cx0 = a.tiles[2 * blockIdx.x] * JX, cy0 = a.tiles[2 * blockIdx.x + 1] * JY;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_expect_tx(&bar, (uint32_t)(HX * HY * sizeof(T) + (PRO ? HY * CLX + UCY * UCX * sizeof(T) : 0)));
    tma_load_3d(tile, &tin, &bar, cx0, cy0, 0);
    if (PRO) {
      tma_load_2d(ctile, &tcls, &bar, cx0, cy0);
      tma_load_3d(uct, &tuc, &bar, cx0 / 2, cy0 / 2 + 1, 0);
    }
  }
  const int x = threadIdx.x & 63, y0 = (threadIdx.x >> 6) * 8;
  const int i = cx0 + x;
  uint8_t cv[8];
  T rv[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int j = cy0 + y0 + k;
    const long p = (long)(j + 2) * a.pitch + (i + 2);
    const bool in = i < a.nx && j < a.ny;
    if (!PRO) cv[k] = in ? a.cls[p] : (uint8_t)0;
    rv[k] = in ? a.r[p] : (T)0;
  }
  bool ok = tile_wait(&bar, a.err);
  if (PRO) {
    // every thread passes the barrier; the staged cell (y, x) has its parent at
    // (y / 2, x / 2 + 1) of the coarse box
    if (ok)
      for (int idx = threadIdx.x; idx < HY * HX; idx += blockDim.x) {
        const int y = idx / HX, xx = idx - y * HX;
        if (ctile[y * CLX + xx] == 1) tile[idx] += uct[(y >> 1) * UCX + (xx >> 1) + 1];
      }
    ok = __syncthreads_and(ok);
#pragma unroll
    for (int k = 0; k < 8; ++k) cv[k] = ctile[(y0 + k + 2) * CLX + x + 2];
  }
  if (!ok || i >= a.nx) return;
  T w[5][5];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int b = 0; b < 5; ++b) w[q][b] = tile[(y0 + q) * HX + x + b];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
#pragma unroll
    for (int b = 0; b < 5; ++b) w[4][b] = tile[(y0 + k + 4) * HX + x + b];
    if (cv[k] == 1) {
      T acc = 0;
#pragma unroll
      for (int q = 0; q < 5; ++q)
#pragma unroll
        for (int b = 0; b < 5; ++b) {
          if (!CROSS && q != 2 && b != 2) continue;
          acc += a.S.w[q * 5 + b] * w[q][b];
        }
      const long p = (long)(cy0 + y0 + k + 2) * a.pitch + (i + 2);
      a.u_new[p] = w[2][2] + a.S.omega_d * (rv[k] - acc);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int b = 0; b < 5; ++b) w[q][b] = w[q + 1][b];
  }
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// SMO-2 blocks of a sweep as their own kernel (a parallel branch beside the regular-cell
// sweep): the block's rows of inv(L22[ext, ext]) arrive in shared memory by one bulk copy
// while the residuals of the extended rows are computed from the old iterate.
template <typename T>
__global__ void __launch_bounds__(256) k_blocks(SweepArgs<T> a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ T part[8][32];
  a.u_old += (long)blockIdx.y * a.bs;      // right-hand side blockIdx.y of the batch
  a.u_new += (long)blockIdx.y * a.bs;
  a.r += (long)blockIdx.y * a.bs;
  if (a.uc) a.uc += (long)blockIdx.y * a.bsc;
  const int b = blockIdx.x / a.chunks, chunk = blockIdx.x % a.chunks;
  const int cs = a.blk[4 * b], ce = a.blk[4 * b + 1], es = a.blk[4 * b + 2], ee = a.blk[4 * b + 3];
  const int ne = ee - es, nc = ce - cs;
  const int c0 = chunk * a.rows_per_cta;
  if (c0 >= nc) return;
  T* As = reinterpret_cast<T*>(smem_raw);                       // [ne][nc]
  const uint32_t abytes = (uint32_t)(((long)ne * nc * sizeof(T) + 15) & ~15L);
  T* s = reinterpret_cast<T*>(smem_raw + abytes);               // [ne]
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_expect_tx(&bar, abytes);
    bulk_load(As, a.inv + a.blk_off[b], abytes, &bar);
  }
  for (int e = threadIdx.x; e < ne; e += blockDim.x) {
    const int row = es + e;
    T acc = 0;
    if (a.uc) {
#pragma unroll 15
      for (int k = 0; k < a.W; ++k) {
        const int pq = a.par[(long)k * a.n2 + row];
        T v = a.u_old[a.col[(long)k * a.n2 + row]];
        if (pq >= 0) v += a.uc[pq];
        acc += a.val[(long)k * a.n2 + row] * v;
      }
    } else {
#pragma unroll 15
      for (int k = 0; k < a.W; ++k) acc += a.val[(long)k * a.n2 + row] * a.u_old[a.col[(long)k * a.n2 + row]];
    }
    s[e] = a.r[a.cell[row]] - acc;
  }
  const bool ok = tile_wait(&bar, a.err);
  __syncthreads();
  if (!ok) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int cend = min(nc, c0 + a.rows_per_cta);
  for (int cb = c0; cb < cend; cb += 32) {
    const int c = cb + lane;
    T acc = 0;
    if (c < cend)
      for (int e = warp; e < ne; e += nw) acc += As[e * nc + c] * s[e];
    part[warp][lane] = acc;
    __syncthreads();
    if (warp == 0 && c < cend) {
      T tot = 0;
      for (int w = 0; w < nw; ++w) tot += part[w][lane];
      const long q = a.cell[cs + c];
      a.u_new[q] = a.u_old[q] + tot;
    }
    __syncthreads();
  }
}

// TMA-staged residual + restriction: a 64 x 32 tile of fine cells (with its halo) gives the
// residuals of all its cells in shared memory, then the 32 x 16 coarse cells it covers get
// the volume-weighted restriction and a zero coarse iterate.  The fitted rows of the tile's
// irregular cells (listed per tile: row and position in the tile) are evaluated first, one
// row per thread, while the tile copy is in flight; the regular cells then take the
// stencil from the staged tile.  The cell volumes are read once, in the coarse phase.
template <typename T, bool CROSS>
__global__ void __launch_bounds__(256, 4) k_restrict_tma(const __grid_constant__ CUtensorMap tin,
                                                         const int32_t* __restrict__ tiles, int nxf, int nyf,
                                                         int pitchf, const uint8_t* __restrict__ clsf,
                                                         const T* __restrict__ volf, const int32_t* __restrict__ rr_off,
                                                         const int32_t* __restrict__ rr, int n2, int W,
                                                         const int32_t* __restrict__ irr_cell,
                                                         const int32_t* __restrict__ col, const T* __restrict__ val,
                                                         const T* __restrict__ u, const T* __restrict__ r, int nxc,
                                                         int nyc, int pitchc, const uint8_t* __restrict__ clsc,
                                                         T* __restrict__ rc, T* __restrict__ uc, Stencil<T> S,
                                                         int* __restrict__ err) {
  pdl_enter();
  __shared__ __align__(128) T tile[HY * HX];
  __shared__ T res[JY][JX];      // residual of every fine cell of the tile (0 on empty cells)
  __shared__ __align__(8) uint64_t bar;
  const int cx0 = tiles[2 * blockIdx.x] * JX, cy0 = tiles[2 * blockIdx.x + 1] * JY;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_expect_tx(&bar, (uint32_t)(HX * HY * sizeof(T)));
    tma_load_3d(tile, &tin, &bar, cx0, cy0, 0);
  }
  const int k0 = rr_off[blockIdx.x], k1 = rr_off[blockIdx.x + 1];
  for (int k = k0 + (int)threadIdx.x; k < k1; k += blockDim.x) {
    const int row = rr[2 * k], loc = rr[2 * k + 1];
    T acc = 0;
#pragma unroll 15
    for (int m = 0; m < W; ++m) acc += val[(long)m * n2 + row] * u[col[(long)m * n2 + row]];
    res[loc >> 6][loc & 63] = r[irr_cell[row]] - acc;
  }
  const int x = threadIdx.x & 63, y0 = (threadIdx.x >> 6) * 8;
  const int i = cx0 + x;
  uint8_t cv[8];
  T rv[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int j = cy0 + y0 + k;
    const long p = (long)(j + 2) * pitchf + (i + 2);
    const bool in = i < nxf && j < nyf;
    cv[k] = in ? clsf[p] : (uint8_t)0;
    rv[k] = in ? r[p] : (T)0;
  }
  const bool ok = tile_wait(&bar, err);
  if (ok) {
    T w[5][5];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int b = 0; b < 5; ++b) w[q][b] = tile[(y0 + q) * HX + x + b];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
#pragma unroll
      for (int b = 0; b < 5; ++b) w[4][b] = tile[(y0 + k + 4) * HX + x + b];
      if (cv[k] == 1) {
        T acc = 0;
#pragma unroll
        for (int q = 0; q < 5; ++q)
#pragma unroll
          for (int b = 0; b < 5; ++b) {
            if (!CROSS && q != 2 && b != 2) continue;
            acc += S.w[q * 5 + b] * w[q][b];
          }
        res[y0 + k][x] = rv[k] - acc;
      } else if (cv[k] == 0) {
        res[y0 + k][x] = (T)0;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int b = 0; b < 5; ++b) w[q][b] = w[q + 1][b];
    }
  }
  if (!__syncthreads_and(ok)) return;
  // 32 x 16 coarse cells, two per thread
  for (int t = threadIdx.x; t < (JX / 2) * (JY / 2); t += blockDim.x) {
    const int ci = t % (JX / 2), cj = t / (JX / 2);
    const int I = cx0 / 2 + ci, J = cy0 / 2 + cj;
    if (I >= nxc || J >= nyc) continue;
    const long pc = (long)(J + 2) * pitchc + (I + 2);
    if (clsc[pc] == 0) continue;
    const long f0 = (long)(2 * J + 2) * pitchf + (2 * I + 2);
    const T v0 = volf[f0], v1 = volf[f0 + 1], v2 = volf[f0 + pitchf], v3 = volf[f0 + pitchf + 1];
    const T s = v0 * res[2 * cj][2 * ci] + v1 * res[2 * cj][2 * ci + 1] + v2 * res[2 * cj + 1][2 * ci] +
                v3 * res[2 * cj + 1][2 * ci + 1];
    const T sv = v0 + v1 + v2 + v3;
    rc[pc] = sv > (T)0 ? (T)4 * s / sv : (T)0;
    uc[pc] = (T)0;
  }
}

// residual + restriction in one launch: every child's residual is computed here (regular
// children by the stencil, irregular children by their fitted row through rowmap)
template <typename T, bool CROSS>
__global__ void k_restrict_rows(int nxc, int nyc, int pitchc, int pitchf, const uint8_t* __restrict__ clsc,
                                const uint8_t* __restrict__ clsf, const T* __restrict__ volf,
                                const int32_t* __restrict__ rowmap, int n2, int W, const int32_t* __restrict__ col,
                                const T* __restrict__ val, const T* __restrict__ u, const T* __restrict__ r,
                                T* __restrict__ rc, T* __restrict__ uc, Stencil<T> S, long bs, long bsc) {
  pdl_enter();
  u += blockIdx.z * bs;       // right-hand side blockIdx.z of the batch
  r += blockIdx.z * bs;
  rc += blockIdx.z * bsc;
  uc += blockIdx.z * bsc;
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
    T Lu;
    if (c == 1) {
      Lu = stencil_apply<T, CROSS>(u, q, pitchf, S);
    } else {
      const int row = rowmap[q];
      Lu = 0;
#pragma unroll 15
      for (int m = 0; m < W; ++m) Lu += val[(long)m * n2 + row] * u[col[(long)m * n2 + row]];
    }
    T v = volf[q];
    s += v * (r[q] - Lu);
    sv += v;
  }
  rc[pc] = sv > (T)0 ? (T)4 * s / sv : (T)0;
  uc[pc] = (T)0;
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

// SMO-2 fused with the residual of the fitted rows.  Rows are numbered in the boundary
// order, so block b owns the contiguous core rows [cs, ce) and reads the extended range
// [es, ee).  The residual of a row uses the new regular values (u_new, written by SMO-1;
// flagged columns) and the old irregular values (u_old); the core rows then get
// u_new = u_old + inv(L22[ext, ext])[core, :] res[ext].  Every irregular cell is the core of
// exactly one block and no kernel writes what it reads.  One CTA of 256 threads per block
// (blockIdx.y splits the core rows only for the single exact block of a small level).
template <typename T>
__global__ void __launch_bounds__(256) k_block_fused(const int32_t* __restrict__ blk,
                                                     const int64_t* __restrict__ blk_off, const T* __restrict__ inv,
                                                     int n2, int W, const int32_t* __restrict__ cell,
                                                     const int32_t* __restrict__ colf, const T* __restrict__ val,
                                                     const T* __restrict__ r, const T* __restrict__ u_old,
                                                     T* __restrict__ u_new, int rows_per_cta) {
  extern __shared__ unsigned char smem_raw[];
  T* s = reinterpret_cast<T*>(smem_raw);
  __shared__ T part[8][32];
  const int b = blockIdx.x;
  const int cs = blk[4 * b], ce = blk[4 * b + 1], es = blk[4 * b + 2], ee = blk[4 * b + 3];
  const int ne = ee - es, nc = ce - cs;
  const int c0 = blockIdx.y * rows_per_cta;
  if (c0 >= nc) return;
  for (int e = threadIdx.x; e < ne; e += blockDim.x) {
    const int row = es + e;
    T acc = 0;
#pragma unroll 15
    for (int k = 0; k < W; ++k) {
      const int f = colf[(long)k * n2 + row];
      const int q = f & 0x7fffffff;
      acc += val[(long)k * n2 + row] * (f < 0 ? u_new[q] : u_old[q]);
    }
    s[e] = r[cell[row]] - acc;
  }
  __syncthreads();
  const T* A = inv + blk_off[b];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int cend = min(nc, c0 + rows_per_cta);
  for (int cb = c0; cb < cend; cb += 32) {
    const int c = cb + lane;
    T acc = 0;
    if (c < cend)
      for (int e = warp; e < ne; e += nw) acc += A[(long)e * nc + c] * s[e];
    part[warp][lane] = acc;
    __syncthreads();
    if (warp == 0 && c < cend) {
      T tot = 0;
      for (int w = 0; w < nw; ++w) tot += part[w][lane];
      const long q = cell[cs + c];
      u_new[q] = u_old[q] + tot;
    }
    __syncthreads();
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
                          int pitch, int pitchc, const T* __restrict__ uc, T* __restrict__ u, long bs, long bsc) {
  pdl_enter();
  uc += blockIdx.y * bsc;     // right-hand side blockIdx.y of the batch
  u += blockIdx.y * bs;
  int i, j;
  long p;
  if (!tile_cell(tiles, nx, ny, pitch, i, j, p)) return;
  if (cls[p] != 1) return;
  u[p] += uc[(long)(j / 2 + 2) * pitchc + (i / 2 + 2)];
}

// bottom solve: u[cell_k] = sum_c inv[c][k] r[cell_c]
// The bottom solve u = inv(L_bottom) r split over a thread-block cluster of BOTTOM_SPLIT
// CTAs: CTA q of the cluster takes columns [q n / S, (q + 1) n / S) of the 32 rows of its row
// block, warps split those columns, and the cluster's rank 0 adds the S partial sums through
// distributed shared memory in rank order (the same order every run).  Both cluster barriers
// are passed by every thread of every CTA.
constexpr int BOTTOM_SPLIT = 8;

__device__ __forceinline__ unsigned bottom_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ void bottom_cluster_sync() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

template <typename T>
__global__ void __launch_bounds__(256) k_bottom_split(int n, const int32_t* __restrict__ cell, const T* __restrict__ inv,
                                                      const T* __restrict__ r, T* __restrict__ u, long bs) {
  __shared__ T part[8][32];
  __shared__ T tot[32];
  const unsigned q = bottom_rank();
  const int rowblk = blockIdx.x / BOTTOM_SPLIT;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int k = rowblk * 32 + lane;
  const int c0 = (int)((long)n * q / BOTTOM_SPLIT), c1 = (int)((long)n * (q + 1) / BOTTOM_SPLIT);
  // this CTA's part of the inverse and the cells of its columns, while the previous launch
  // drains (a warp's 32 rows of one column are one line)
  if (k < n)
    for (int c = c0 + warp; c < c1; c += 8) prefetch_l1(inv + (long)c * n + k);
  for (int c = c0 + (int)threadIdx.x * 32; c < c1; c += (int)blockDim.x * 32) prefetch_l1(cell + c);
  pdl_enter();
  r += blockIdx.y * bs;       // right-hand side blockIdx.y of the batch
  u += blockIdx.y * bs;
  T acc = 0;
  if (k < n)
    for (int c = c0 + warp; c < c1; c += 8) acc += inv[(long)c * n + k] * r[cell[c]];
  part[warp][lane] = acc;
  __syncthreads();
  if (warp == 0) {
    T s = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) s += part[w][lane];
    tot[lane] = s;
  }
  bottom_cluster_sync();          // every CTA's tot is written
  if (q == 0 && warp == 0) {
    uint32_t local = (uint32_t)__cvta_generic_to_shared(&tot[lane]);
    T s = 0;
    for (unsigned p = 0; p < BOTTOM_SPLIT; ++p) {
      uint32_t remote;
      asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(p));
      T v;
      if constexpr (sizeof(T) == 8) {
        asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(remote) : "memory");
      } else {
        asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(remote) : "memory");
      }
      s += v;
    }
    if (k < n) u[cell[k]] = s;
  }
  bottom_cluster_sync();          // the other CTAs keep their shared memory until rank 0 has read it
}

template <typename T>
__global__ void k_bottom(int n, const int32_t* __restrict__ cell, const T* __restrict__ inv,
                         const T* __restrict__ r, T* __restrict__ u, long bs) {
  pdl_enter();
  r += blockIdx.y * bs;       // right-hand side blockIdx.y of the batch
  u += blockIdx.y * bs;
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

// user layout <- padded, scaled; the empty cells of dst are set to 0, or with KEEP left as
// they are (a destination across the host link gets only the cells that hold unknowns)
template <typename TS, bool KEEP = false>
__global__ void k_unpack(int nx, int ny, int pitch, const uint8_t* __restrict__ cls, const TS* __restrict__ src,
                         double* __restrict__ dst, double scale) {
  int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= nx) return;
  long p = (long)(j + 2) * pitch + (i + 2);
  if (cls[p] != 0) dst[(long)j * nx + i] = scale * (double)src[p];
  else if (!KEEP) dst[(long)j * nx + i] = 0.0;
}

// k_pack and k_unpack over the level's active 32 x 8 tiles (every non-empty cell lies in one;
// on a domain that covers a fraction of the box the rest of the grid is not visited).  The
// tiled unpack writes the non-empty cells only: a caller that wants 0 on the empty cells
// clears the destination first.
template <typename TD, typename TS>
__global__ void k_pack_tiles(const int32_t* __restrict__ tiles, int nx, int ny, int pitch, const uint8_t* __restrict__ cls,
                             const TS* __restrict__ src, TD* __restrict__ dst, double scale) {
  const int i = tiles[2 * blockIdx.x] * TX + threadIdx.x, j = tiles[2 * blockIdx.x + 1] * TY + threadIdx.y;
  if (i >= nx || j >= ny) return;
  const long p = (long)(j + 2) * pitch + (i + 2);
  if (cls[p] != 0) dst[p] = (TD)(scale * (double)src[(long)j * nx + i]);
}

template <typename TS>
__global__ void k_unpack_tiles(const int32_t* __restrict__ tiles, int nx, int ny, int pitch,
                               const uint8_t* __restrict__ cls, const TS* __restrict__ src, double* __restrict__ dst,
                               double scale) {
  const int i = tiles[2 * blockIdx.x] * TX + threadIdx.x, j = tiles[2 * blockIdx.x + 1] * TY + threadIdx.y;
  if (i >= nx || j >= ny) return;
  const long p = (long)(j + 2) * pitch + (i + 2);
  if (cls[p] != 0) dst[(long)j * nx + i] = scale * (double)src[p];
}

// max |x| over the non-empty cells of the active 32 x 8 tiles (as k_absmax), CTAs striding
// over the tiles; right-hand side blockIdx.y of a batch at stride bs
template <typename T>
__global__ void k_absmax_tiles(const int32_t* __restrict__ tiles, int ntiles, int nx, int ny, int pitch,
                               const uint8_t* __restrict__ cls, const T* __restrict__ x,
                               unsigned long long* __restrict__ out, long bs) {
  pdl_enter();
  x += blockIdx.y * bs;
  out += blockIdx.y;
  double m = 0.0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int i = tiles[2 * t] * TX + threadIdx.x, j = tiles[2 * t + 1] * TY + threadIdx.y;
    if (i < nx && j < ny) {
      const long p = (long)(j + 2) * pitch + (i + 2);
      if (cls[p] != 0) {
        double v = fabs((double)x[p]);
        if (!(v <= 1.7976931348623157e308)) v = __longlong_as_double(0x7ff0000000000000ULL);   // NaN -> Inf
        m = fmax(m, v);
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (threadIdx.x == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
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
                         unsigned long long* __restrict__ out, long bs) {
  pdl_enter();
  x += blockIdx.y * bs;       // right-hand side blockIdx.y of the batch: its own word
  out += blockIdx.y;
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
  pdl_enter();
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < n; p += (long)gridDim.x * blockDim.x)
    if (cls[p] != 0) u[p] += (double)e[p];
}
__global__ void k_to_float(long n, const double* __restrict__ a, float* __restrict__ b) {
  pdl_enter();
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
