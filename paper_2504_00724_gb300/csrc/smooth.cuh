// One block-Jacobi smoothing sweep of a level (SMO-1 on the regular cells and the SMO-2
// overlapping-block corrections of the irregular cells, both from the old iterate, Sec. 4.1)
// as one persistent launch.
//
// Work items: the SMO-2 blocks first, then the 64 x 32 cell tiles with a regular cell.  CTA c
// takes items c, c + G, c + 2G, ... (G = grid size, a multiple of the SM count where the
// level is large).  Every item's operands arrive in one of two shared-memory stages, so the
// copy of item k + 1 is in flight while item k computes:
//   tile item:  the 68 x 36 halo tile of u, the 68 x 32 box of r over the tile's rows and the
//               80 x 36 class bytes (one 2-D TMA box each; x origin 64a, 16-byte aligned),
//               and with PRO the 36 x 18 box of the coarse iterate under the tile;
//   block item: the block's rows of inv(L22[ext, ext]) by one bulk copy (cp.async.bulk); the
//               residuals of its extended rows are gathered from global memory meanwhile.
// With PRO the sweep is the first post-smoothing sweep of Alg. 2 and reads u + P uc, the
// coarse correction added to regular cells only (Sec. 4.1).  A level's first sweep may start
// from a zero iterate (zero_u: no iterate copied or gathered), and the last level-0 sweep of
// an outer iteration may add its new values to the FP64 solution (uhat).
// Before the grid dependency wait each CTA does what depends on no earlier launch: copy
// barriers, prefetches of its blocks' fitted rows, and the copies of its first two items'
// static parts (inverse rows, class bytes); the iterate and r follow the wait.
// Waits are bounded by the SM clock; a wait that runs out sets the error word, waits (again
// bounded) for every copy still in flight, and the CTA leaves, all threads together.
#pragma once

#include "kernels.cuh"

namespace ccm {
namespace dev {

template <typename T>
struct SmoothArgs {
  SweepArgs<T> a;      // level arrays, stencil, iterates, blocks (chunks == 1)
  int nbi;             // block items (= a.nblk)
  int nitems;          // nbi + a.ntiles
  uint32_t stage;      // bytes per stage (multiple of 128)
  int max_ext;         // most extended rows of a block (the per-row scratch after the stages)
};


// two adjacent values of T (8 or 16 bytes, aligned)
template <typename T> struct Pair;
template <> struct Pair<float> { using type = float2; };
template <> struct Pair<double> { using type = double2; };

// w[0..5] = row[0..5] as three aligned pair loads (row at an even element offset)
template <typename T>
__device__ __forceinline__ void load_six(const T* row, T (&w)[6]) {
  using V2 = typename Pair<T>::type;
  const V2 a = *reinterpret_cast<const V2*>(row);
  const V2 b = *reinterpret_cast<const V2*>(row + 2);
  const V2 c = *reinterpret_cast<const V2*>(row + 4);
  w[0] = a.x;
  w[1] = a.y;
  w[2] = b.x;
  w[3] = b.y;
  w[4] = c.x;
  w[5] = c.y;
}

// offsets inside a stage of a tile item
template <typename T>
struct TileStage {
  static constexpr uint32_t al(uint32_t b) { return (b + 127u) & ~127u; }
  static constexpr uint32_t u_bytes = HY * HX * sizeof(T);
  static constexpr uint32_t r_bytes = JY * HX * sizeof(T);
  static constexpr uint32_t c_bytes = HY * CLX;
  static constexpr uint32_t uc_bytes = UCY * UCX * sizeof(T);
  static constexpr uint32_t r_off = al(u_bytes);
  static constexpr uint32_t c_off = r_off + al(r_bytes);
  static constexpr uint32_t uc_off = c_off + al(c_bytes);
  static constexpr uint32_t bytes(bool pro) { return pro ? uc_off + uc_bytes : c_off + c_bytes; }
};

__device__ __forceinline__ bool wait_parity(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (clock64() - t0 < TMA_WAIT_CYCLES)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// The copy of an item into stage st, completing on bar.  part 0: all of it; part 1: what
// does not depend on the previous launch (a block's inverse rows; a tile's class bytes, with
// the byte count of the whole tile), issued before the grid dependency wait; part 2: the rest
// of a tile (iterate, right-hand side, coarse iterate), after it.
template <typename T, bool PRO>
__device__ __forceinline__ void smooth_issue(const SmoothArgs<T>& A, const CUtensorMap* tin, const CUtensorMap* tr,
                                             const CUtensorMap* tcls, const CUtensorMap* tuc, int item,
                                             unsigned char* st, uint64_t* bar, int part = 0) {
  const int z = blockIdx.y;      // right-hand side of the batch
  const SweepArgs<T>& a = A.a;
  if (item < A.nbi) {
    if (part == 2) return;
    const int b = item;
    const int nc = a.blk[4 * b + 1] - a.blk[4 * b], ne = a.blk[4 * b + 3] - a.blk[4 * b + 2];
    const uint32_t abytes = (uint32_t)(((long)ne * nc * sizeof(T) + 15) & ~15L);
    mbar_expect_tx(bar, abytes);
    bulk_load(st, a.inv + a.blk_off[b], abytes, bar);
  } else {
    using S = TileStage<T>;
    const int t = item - A.nbi;
    const int cx0 = a.tiles[2 * t] * JX, cy0 = a.tiles[2 * t + 1] * JY;
    const bool no_u = !PRO && sizeof(T) == 4 && a.zero_u;     // the old iterate is 0
    if (part != 2) {
      mbar_expect_tx(bar, (no_u ? 0u : S::u_bytes) + S::r_bytes + S::c_bytes + (PRO ? S::uc_bytes : 0));
      tma_load_2d(st + S::c_off, tcls, bar, cx0, cy0);
    }
    if (part != 1) {
      if (!no_u) tma_load_3d(st, tin, bar, cx0, cy0, z);
      tma_load_3d(st + S::r_off, tr, bar, cx0, cy0 + 2, z);
      if (PRO) tma_load_3d(st + S::uc_off, tuc, bar, cx0 / 2, cy0 / 2 + 1, z);
    }
  }
}

// SMO-2 residuals of block b's extended rows from u_old (u_old + P uc with PRO) into sres,
// and each row's cell and old value (an irregular cell: no coarse correction) into scell and
// sold for the update of the core rows; the block's core start, core size and extended size
// come back, the core's first row at extended row cs - es.  CG: u_old is read through L2
// only (iterates that other CTAs of the same launch wrote).
template <typename T, bool PRO, bool CG>
__device__ __forceinline__ void block_residuals(const SweepArgs<T>& a, int b, const T* __restrict__ u_old,
                                                const T* __restrict__ rhs, const T* __restrict__ ucs, T* sres,
                                                T* sold, int* scell, int& cs, int& nc, int& ne, int& es) {
  cs = a.blk[4 * b];
  nc = a.blk[4 * b + 1] - cs;
  es = a.blk[4 * b + 2];
  ne = a.blk[4 * b + 3] - es;
  for (int e = threadIdx.x; e < ne; e += blockDim.x) {
    const int row = es + e;
    const int q = a.cell[row];
    if (!PRO && sizeof(T) == 4 && a.zero_u) {   // the old iterate is 0: the residual is r
      sres[e] = rhs[q];
      sold[e] = (T)0;
      scell[e] = q;
      continue;
    }
    T acc = 0;
#pragma unroll 15
    for (int m = 0; m < a.W; ++m) {
      const int cq = a.col[(long)m * a.n2 + row];
      T v = CG ? __ldcg(u_old + cq) : u_old[cq];
      if (PRO) {
        const int pq = a.par[(long)m * a.n2 + row];
        if (pq >= 0) v += ucs[pq];
      }
      acc += a.val[(long)m * a.n2 + row] * v;
    }
    sres[e] = rhs[q] - acc;
    sold[e] = CG ? __ldcg(u_old + q) : u_old[q];
    scell[e] = q;
  }
}

// u_new = u_old + inv(L22[ext, ext]) sres on the block's core cells; As = the staged rows
// [ne][nc] of the inverse, columns over lanes, extended rows over warps; the core cells and
// their old values from scell and sold (no global round trip before the stores)
template <typename T>
__device__ __forceinline__ void block_apply(const T* As, const T* sres, const T* sold, const int* scell, int c0,
                                            int nc, int ne, T* __restrict__ u_new, double* __restrict__ uhat,
                                            T (*part)[32]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int cb = 0; cb < nc; cb += 32) {
    const int c = cb + lane;
    T acc = 0;
    if (c < nc)
      for (int e = warp; e < ne; e += 8) acc += As[e * nc + c] * sres[e];
    part[warp][lane] = acc;
    __syncthreads();
    if (warp == 0 && c < nc) {
      T tot = 0;
#pragma unroll
      for (int w = 0; w < 8; ++w) tot += part[w][lane];
      const int q = scell[c0 + c];
      const T v = sold[c0 + c] + tot;
      u_new[q] = v;
      if (uhat) uhat[q] += (double)v;
    }
    __syncthreads();
  }
}

// SMO-1 on the regular cells of a staged 64 x 32 tile (halo box of u, box of r and class bytes
// at the TileStage offsets of st; with PRO the coarse box too, whose parent values are first
// added to the staged regular cells: the sweep then reads u + P uc)
template <typename T, bool CROSS, bool PRO>
__device__ __forceinline__ void tile_sweep(const SweepArgs<T>& a, unsigned char* st, int cx0, int cy0,
                                           T* __restrict__ u_new, double* __restrict__ uhat) {
  using S = TileStage<T>;
  T* tile = reinterpret_cast<T*>(st);
  const T* rt = reinterpret_cast<const T*>(st + S::r_off);
  const uint8_t* ct = st + S::c_off;
  if (PRO) {
    // staged cell (y, x) has its parent at (y / 2, x / 2 + 1) of the coarse box; four cells
    // (one 32-bit word of class bytes, two parents, two aligned pairs of the tile) per step,
    // the tile's 36 x 17 quads spread over all threads
    using P2 = typename Pair<T>::type;
    const T* uct = reinterpret_cast<const T*>(st + S::uc_off);
    for (int q = threadIdx.x; q < HY * (HX / 4); q += blockDim.x) {
      const int y = q / (HX / 4), xq = q - y * (HX / 4), x0 = 4 * xq;
      const uint32_t c4 = *reinterpret_cast<const uint32_t*>(ct + y * CLX + x0);
      const T p0 = uct[(y >> 1) * UCX + 2 * xq + 1], p1 = uct[(y >> 1) * UCX + 2 * xq + 2];
      P2* tr = reinterpret_cast<P2*>(tile + y * HX + x0);
      P2 v0 = tr[0], v1 = tr[1];
      if ((c4 & 0xffu) == 1u) v0.x += p0;
      if (((c4 >> 8) & 0xffu) == 1u) v0.y += p0;
      if (((c4 >> 16) & 0xffu) == 1u) v1.x += p1;
      if ((c4 >> 24) == 1u) v1.y += p1;
      tr[0] = v0;
      tr[1] = v1;
    }
    __syncthreads();
  }
  if constexpr (sizeof(T) == 8) {
    // FP64: one cell column of eight rows per thread (the paired form below spills).  FP64
    // issue bounds this loop, so with the mixed term the stencil is taken in factored form: the
    // x-derivative of each entering row (4 FMA) and 13 FMA per cell, against 25
    const int x = threadIdx.x & 63, y0 = (threadIdx.x >> 6) * 8;
    const int i = cx0 + x;
    if (i < a.nx) {
      T w[5][5], D[5];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
#pragma unroll
        for (int b = 0; b < 5; ++b) w[q][b] = tile[(y0 + q) * HX + x + b];
        if (CROSS) D[q] = a.S.gx[0] * w[q][0] + a.S.gx[1] * w[q][1] + a.S.gx[3] * w[q][3] + a.S.gx[4] * w[q][4];
      }
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) {
#pragma unroll
        for (int b = 0; b < 5; ++b) w[4][b] = tile[(y0 + kk + 4) * HX + x + b];
        if (CROSS) D[4] = a.S.gx[0] * w[4][0] + a.S.gx[1] * w[4][1] + a.S.gx[3] * w[4][3] + a.S.gx[4] * w[4][4];
        if (ct[(y0 + kk + 2) * CLX + x + 2] == 1) {
          T acc = 0;
          if (CROSS) {
            acc = a.S.cc * w[2][2];
            acc = fma(a.S.lx[0], w[2][0], acc);
            acc = fma(a.S.lx[1], w[2][1], acc);
            acc = fma(a.S.lx[3], w[2][3], acc);
            acc = fma(a.S.lx[4], w[2][4], acc);
            acc = fma(a.S.ly[0], w[0][2], acc);
            acc = fma(a.S.ly[1], w[1][2], acc);
            acc = fma(a.S.ly[3], w[3][2], acc);
            acc = fma(a.S.ly[4], w[4][2], acc);
            acc = fma(a.S.gy[0], D[0], acc);
            acc = fma(a.S.gy[1], D[1], acc);
            acc = fma(a.S.gy[3], D[3], acc);
            acc = fma(a.S.gy[4], D[4], acc);
          } else {
#pragma unroll
            for (int q = 0; q < 5; ++q)
#pragma unroll
              for (int b = 0; b < 5; ++b) {
                if (q != 2 && b != 2) continue;
                acc += a.S.w[q * 5 + b] * w[q][b];
              }
          }
          const long p = (long)(cy0 + y0 + kk + 2) * a.pitch + (i + 2);
          u_new[p] = w[2][2] + a.S.omega_d * (rt[(y0 + kk) * HX + x + 2] - acc);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
#pragma unroll
          for (int b = 0; b < 5; ++b) w[q][b] = w[q + 1][b];
          if (CROSS) D[q] = D[q + 1];
        }
      }
    }
  } else {
    // FP32: two adjacent cells (x0, x0 + 1) in four rows per thread: each staged row is read
    // as three aligned pairs (x0 - 2 .. x0 + 3) and serves both cells' stencils, and the
    // class bytes, right-hand sides and new values move in pairs
    using V2 = typename Pair<T>::type;
    const int x0 = 2 * (threadIdx.x & 31), y0 = (threadIdx.x >> 5) * 4;
    const int i0 = cx0 + x0;
    // the new values of row kk's pair: into u_new, and added to u_hat when the sweep folds in
    // the outer iteration's update
    auto put = [&](int kk, T v0, T v1, uint32_t c2) {
      const bool g0 = (c2 & 0xffu) == 1u, g1 = (c2 >> 8) == 1u && i0 + 1 < a.nx;
      const long p = (long)(cy0 + y0 + kk + 2) * a.pitch + (i0 + 2);
      if (g0 && g1) {
        V2 o;
        o.x = v0;
        o.y = v1;
        *reinterpret_cast<V2*>(u_new + p) = o;
      } else {
        if (g0) u_new[p] = v0;
        if (g1) u_new[p + 1] = v1;
      }
      if (uhat) {
        if (g0) uhat[p] += (double)v0;
        if (g1) uhat[p + 1] += (double)v1;
      }
    };
    if (!PRO && a.zero_u) {
      // the old iterate is 0 (its tile was not copied): u_new = omega_d r on the regular cells
      if (i0 < a.nx)
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint32_t c2 = *reinterpret_cast<const uint16_t*>(ct + (y0 + kk + 2) * CLX + x0 + 2);
          const V2 r2 = *reinterpret_cast<const V2*>(rt + (y0 + kk) * HX + x0 + 2);
          put(kk, a.S.omega_d * r2.x, a.S.omega_d * r2.y, c2);
        }
      return;
    }
    if (i0 < a.nx) {
      T w[5][6];
#pragma unroll
      for (int q = 0; q < 4; ++q) load_six(tile + (y0 + q) * HX + x0, w[q]);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        load_six(tile + (y0 + kk + 4) * HX + x0, w[4]);
        T acc0 = 0, acc1 = 0;
#pragma unroll
        for (int q = 0; q < 5; ++q)
#pragma unroll
          for (int b = 0; b < 5; ++b) {
            if (!CROSS && q != 2 && b != 2) continue;
            acc0 += a.S.w[q * 5 + b] * w[q][b];
            acc1 += a.S.w[q * 5 + b] * w[q][b + 1];
          }
        const uint32_t c2 = *reinterpret_cast<const uint16_t*>(ct + (y0 + kk + 2) * CLX + x0 + 2);
        const V2 r2 = *reinterpret_cast<const V2*>(rt + (y0 + kk) * HX + x0 + 2);
        put(kk, w[2][2] + a.S.omega_d * (r2.x - acc0), w[2][3] + a.S.omega_d * (r2.y - acc1), c2);
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int b = 0; b < 6; ++b) w[q][b] = w[q + 1][b];
      }
    }
  }
}

template <typename T, bool CROSS, bool PRO>
__global__ void __launch_bounds__(256, 3) k_smooth(const __grid_constant__ CUtensorMap tin,
                                                const __grid_constant__ CUtensorMap tr,
                                                const __grid_constant__ CUtensorMap tcls,
                                                const __grid_constant__ CUtensorMap tuc, SmoothArgs<T> A) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ T part[8][32];
  const SweepArgs<T>& a = A.a;
  // While the previous launch drains: pull the static fitted-row data (columns, coefficients,
  // cells, parents) of this CTA's SMO-2 block items into L1, so that each block's residual
  // gathers need one round trip to the iterate instead of two
  for (int b = blockIdx.x; b < A.nbi; b += gridDim.x) {
    const int es = a.blk[4 * b + 2], ne = a.blk[4 * b + 3] - es;
    for (int e = threadIdx.x; e < ne; e += blockDim.x) {
      const int row = es + e;
      prefetch_l1(a.cell + row);
#pragma unroll 15
      for (int m = 0; m < a.W; ++m) {
        prefetch_l1(a.col + (long)m * a.n2 + row);
        prefetch_l1(a.val + (long)m * a.n2 + row);
        if (PRO && a.par) prefetch_l1(a.par + (long)m * a.n2 + row);
      }
    }
    if (threadIdx.x == 0) prefetch_l1(a.blk_off + b);
  }
  const int G = gridDim.x;
  const int K = (A.nitems - (int)blockIdx.x + G - 1) / G;   // items of this CTA (>= 1)
  // also before the wait: the copy barriers, and the parts of the first two items' copies
  // that no earlier launch writes (the rest follows the wait)
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    smooth_issue<T, PRO>(A, &tin, &tr, &tcls, &tuc, blockIdx.x, smem_raw, &bar[0], 1);
    if (K > 1) smooth_issue<T, PRO>(A, &tin, &tr, &tcls, &tuc, blockIdx.x + G, smem_raw + A.stage, &bar[1], 1);
  }
  __syncthreads();
  pdl_enter();
  // this CTA's right-hand side of the batch (blockIdx.y)
  const long bo = (long)blockIdx.y * a.bs;
  const T* __restrict__ u_old = a.u_old + bo;
  T* __restrict__ u_new = a.u_new + bo;
  double* __restrict__ uhat = a.uhat ? a.uhat + bo : nullptr;
  const T* __restrict__ rhs = a.r + bo;
  const T* __restrict__ ucs = PRO ? a.uc + (long)blockIdx.y * a.bsc : nullptr;
  // per extended row of a block item: residual, old value, cell (three slots of max_ext)
  const uint32_t slot = (uint32_t)(((long)A.max_ext * sizeof(T) + 15) & ~15L);
  T* sres = reinterpret_cast<T*>(smem_raw + 2 * A.stage);
  T* sold = reinterpret_cast<T*>(smem_raw + 2 * A.stage + slot);
  int* scell = reinterpret_cast<int*>(smem_raw + 2 * A.stage + 2 * slot);
  if (threadIdx.x == 0) {
    smooth_issue<T, PRO>(A, &tin, &tr, &tcls, &tuc, blockIdx.x, smem_raw, &bar[0], 2);
    if (K > 1) smooth_issue<T, PRO>(A, &tin, &tr, &tcls, &tuc, blockIdx.x + G, smem_raw + A.stage, &bar[1], 2);
  }
  for (int k = 0; k < K; ++k) {
    const int item = blockIdx.x + k * G;
    const int sb = k & 1;
    const uint32_t parity = (k >> 1) & 1;
    int cs = 0, nc = 0, ne = 0, es = 0, cx0 = 0, cy0 = 0;
    if (item < A.nbi) {
      block_residuals<T, PRO, false>(a, item, u_old, rhs, ucs, sres, sold, scell, cs, nc, ne, es);
    } else {
      const int t = item - A.nbi;       // the tile's origin, read before the wait
      cx0 = a.tiles[2 * t] * JX;
      cy0 = a.tiles[2 * t + 1] * JY;
    }
    const bool ok = __syncthreads_and(wait_parity(&bar[sb], parity));
    if (!ok) {
      // this copy and the other stage's (if one was issued) must land before the CTA leaves
      wait_parity(&bar[sb], parity);
      if (k + 1 < K) wait_parity(&bar[sb ^ 1], ((k + 1) >> 1) & 1);
      if (threadIdx.x == 0) atomicExch(a.err, 1);
      return;
    }
    if (item < A.nbi) {
      block_apply<T>(reinterpret_cast<const T*>(smem_raw + sb * A.stage), sres, sold, scell, cs - es, nc, ne, u_new,
                     uhat, part);
    } else {
      tile_sweep<T, CROSS, PRO>(a, smem_raw + sb * A.stage, cx0, cy0, u_new, uhat);
    }
    __syncthreads();      // stage sb is free
    if (threadIdx.x == 0 && k + 2 < K) {
      fence_proxy_async();
      smooth_issue<T, PRO>(A, &tin, &tr, &tcls, &tuc, item + 2 * G, (smem_raw + sb * A.stage), &bar[sb]);
    }
  }
}

}  // namespace dev
}  // namespace ccm

namespace ccm {
namespace dev {

// ---- residual + restriction of a level (Alg. 2: the coarse right-hand side and a zero coarse
// iterate) as one persistent launch over the fine 64 x 32 tiles that restriction visits.
// A tile item's halo tile of u, its boxes of r and of the cell volumes (68 x 32 over the
// tile's rows) and its class bytes (80 x 36) arrive by TMA in one of two stages while the
// previous item computes.  The fitted rows of the tile's irregular cells (listed per tile:
// row and position) are gathered from global memory before the wait, and so are the class
// bytes of the coarse cells the thread restricts to; regular cells take the stencil from the
// staged tile; then the 32 x 16 coarse cells get the volume-weighted 2 x 2 sums.
template <typename T>
struct RestrictArgs {
  const int32_t* tiles;
  int ntiles, nxf, nyf, pitchf;
  const int32_t* rr_off;
  const int32_t* rr;
  int n2, W;
  const int32_t* irr_cell;
  const int32_t* col;
  const T* val;
  const T* u;
  const T* r;
  int nxc, nyc, pitchc;
  const uint8_t* clsc;
  T* rc;
  T* uc;
  Stencil<T> S;
  int* err;
  uint32_t stage;
  long bs, bsc;        // batch strides (elements) of the fine and the coarse level arrays
  int nrr;             // the tiles' irregular rows in tile order: (cell, position) pairs, and
  const int32_t* rq;   // the rows' columns and coefficients [W][nrr]
  const int32_t* rq_col;
  const T* rq_val;
};

template <typename T>
struct RestrictStage {
  static constexpr uint32_t al(uint32_t b) { return (b + 127u) & ~127u; }
  static constexpr uint32_t u_bytes = HY * HX * sizeof(T);
  static constexpr uint32_t r_bytes = JY * HX * sizeof(T);
  static constexpr uint32_t c_bytes = HY * CLX;
  static constexpr uint32_t r_off = al(u_bytes);
  static constexpr uint32_t c_off = r_off + al(r_bytes);
  static constexpr uint32_t v_off = c_off + al(c_bytes);
  static constexpr uint32_t bytes = al(v_off + r_bytes);
  static constexpr uint32_t tx = u_bytes + 2 * r_bytes + c_bytes;
};

// the static data of restriction tile t's irregular rows (cell and position pairs, columns
// and coefficients, contiguous in tile order) into L1: k0, k1 = the tile's row range
template <typename T>
__device__ __forceinline__ void prefetch_tile_rows(const RestrictArgs<T>& A, int k0, int k1) {
  for (int q = k0 + 16 * (int)threadIdx.x; q < k1; q += 16 * (int)blockDim.x) {
    prefetch_l1(A.rq + 2 * (long)q);
#pragma unroll 15
    for (int m = 0; m < A.W; ++m) {
      prefetch_l1(A.rq_col + (long)m * A.nrr + q);
      prefetch_l1(A.rq_val + (long)m * A.nrr + q);
    }
  }
}

template <typename T, bool CROSS>
__global__ void __launch_bounds__(256, 3) k_restrict_p(const __grid_constant__ CUtensorMap tin,
                                                       const __grid_constant__ CUtensorMap tr,
                                                       const __grid_constant__ CUtensorMap tcls,
                                                       const __grid_constant__ CUtensorMap tvol, RestrictArgs<T> A) {
  using S = RestrictStage<T>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ T res[JY][JX];      // residual of every fine cell of the tile (0 on empty cells)
  __shared__ __align__(8) uint64_t bar[2];
  const int G = gridDim.x;
  const int K = (A.ntiles - (int)blockIdx.x + G - 1) / G;
  // the first tile's row range and rows while the previous launch drains
  int n0 = A.rr_off[blockIdx.x], n1 = A.rr_off[blockIdx.x + 1];
  prefetch_tile_rows(A, n0, n1);
  // this CTA's right-hand side of the batch (blockIdx.y)
  const int z = blockIdx.y;
  // tile t's copy into stage sb.  part 0: all of it; part 1: the class bytes and volumes,
  // which no launch writes, with the byte count of the whole tile (before the grid
  // dependency wait); part 2: the iterate and the right-hand side (after it)
  auto issue = [&](int t, int sb, int part) {
    unsigned char* st = smem_raw + sb * A.stage;
    const int cx0 = A.tiles[2 * t] * JX, cy0 = A.tiles[2 * t + 1] * JY;
    if (part != 2) {
      mbar_expect_tx(&bar[sb], S::tx);
      tma_load_2d(st + S::c_off, &tcls, &bar[sb], cx0, cy0);
      tma_load_2d(st + S::v_off, &tvol, &bar[sb], cx0, cy0 + 2);
    }
    if (part != 1) {
      tma_load_3d(st, &tin, &bar[sb], cx0, cy0, z);
      tma_load_3d(st + S::r_off, &tr, &bar[sb], cx0, cy0 + 2, z);
    }
  };
  // the copy barriers and the static parts of the first two tiles' copies too
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    issue(blockIdx.x, 0, 1);
    if (K > 1) issue(blockIdx.x + G, 1, 1);
  }
  __syncthreads();
  pdl_enter();
  const T* __restrict__ uf = A.u + (long)z * A.bs;
  const T* __restrict__ rf = A.r + (long)z * A.bs;
  T* __restrict__ rcz = A.rc + (long)z * A.bsc;
  T* __restrict__ ucz = A.uc + (long)z * A.bsc;
  if (threadIdx.x == 0) {
    issue(blockIdx.x, 0, 2);
    if (K > 1) issue(blockIdx.x + G, 1, 2);
  }
  const int x = threadIdx.x & 63, y0 = (threadIdx.x >> 6) * 8;
  for (int k = 0; k < K; ++k) {
    const int t = blockIdx.x + k * G;
    const int sb = k & 1;
    const uint32_t parity = (k >> 1) & 1;
    const int cx0 = A.tiles[2 * t] * JX, cy0 = A.tiles[2 * t + 1] * JY;
    const int k0 = n0, k1 = n1;
    // the next tile's row range: loaded now, used after this tile's stencil
    if (k + 1 < K) {
      n0 = A.rr_off[t + G];
      n1 = A.rr_off[t + G + 1];
    }
    for (int q = k0 + (int)threadIdx.x; q < k1; q += blockDim.x) {
      const int cell = A.rq[2 * q], loc = A.rq[2 * q + 1];
      T acc = 0;
#pragma unroll 15
      for (int m = 0; m < A.W; ++m) acc += A.rq_val[(long)m * A.nrr + q] * uf[A.rq_col[(long)m * A.nrr + q]];
      res[loc >> 6][loc & 63] = rf[cell] - acc;
    }
    // class bytes of this thread's two coarse cells (0 outside the coarse level)
    uint8_t cc[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c = threadIdx.x + h * 256;
      const int I = cx0 / 2 + c % (JX / 2), J = cy0 / 2 + c / (JX / 2);
      cc[h] = (I < A.nxc && J < A.nyc) ? A.clsc[(long)(J + 2) * A.pitchc + (I + 2)] : (uint8_t)0;
    }
    const bool ok = __syncthreads_and(wait_parity(&bar[sb], parity));
    if (!ok) {
      wait_parity(&bar[sb], parity);
      if (k + 1 < K) wait_parity(&bar[sb ^ 1], ((k + 1) >> 1) & 1);
      if (threadIdx.x == 0) atomicExch(A.err, 1);
      return;
    }
    const unsigned char* st = smem_raw + sb * A.stage;
    const T* tile = reinterpret_cast<const T*>(st);
    const T* rt = reinterpret_cast<const T*>(st + S::r_off);
    const uint8_t* ct = st + S::c_off;
    const T* vt = reinterpret_cast<const T*>(st + S::v_off);
    if constexpr (sizeof(T) == 4) {
      // two adjacent cells in four rows per thread, rows read as aligned pairs (as in k_smooth)
      const int x0 = 2 * (threadIdx.x & 31), y1 = (threadIdx.x >> 5) * 4;
      T w[5][6];
#pragma unroll
      for (int q = 0; q < 4; ++q) load_six(tile + (y1 + q) * HX + x0, w[q]);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        load_six(tile + (y1 + kk + 4) * HX + x0, w[4]);
        T acc0 = 0, acc1 = 0;
#pragma unroll
        for (int q = 0; q < 5; ++q)
#pragma unroll
          for (int b = 0; b < 5; ++b) {
            if (!CROSS && q != 2 && b != 2) continue;
            acc0 += A.S.w[q * 5 + b] * w[q][b];
            acc1 += A.S.w[q * 5 + b] * w[q][b + 1];
          }
        const uint32_t c2 = *reinterpret_cast<const uint16_t*>(ct + (y1 + kk + 2) * CLX + x0 + 2);
        const typename Pair<T>::type r2 = *reinterpret_cast<const typename Pair<T>::type*>(rt + (y1 + kk) * HX + x0 + 2);
        const uint32_t cv0 = c2 & 0xffu, cv1 = c2 >> 8;
        if (cv0 == 1u) res[y1 + kk][x0] = r2.x - acc0;
        else if (cv0 == 0u) res[y1 + kk][x0] = (T)0;
        if (cv1 == 1u) res[y1 + kk][x0 + 1] = r2.y - acc1;
        else if (cv1 == 0u) res[y1 + kk][x0 + 1] = (T)0;
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int b = 0; b < 6; ++b) w[q][b] = w[q + 1][b];
      }
    } else {
      // FP64 (one column per thread), with the mixed term in factored form as in tile_sweep
      T w[5][5], D[5];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
#pragma unroll
        for (int b = 0; b < 5; ++b) w[q][b] = tile[(y0 + q) * HX + x + b];
        if (CROSS) D[q] = A.S.gx[0] * w[q][0] + A.S.gx[1] * w[q][1] + A.S.gx[3] * w[q][3] + A.S.gx[4] * w[q][4];
      }
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) {
#pragma unroll
        for (int b = 0; b < 5; ++b) w[4][b] = tile[(y0 + kk + 4) * HX + x + b];
        if (CROSS) D[4] = A.S.gx[0] * w[4][0] + A.S.gx[1] * w[4][1] + A.S.gx[3] * w[4][3] + A.S.gx[4] * w[4][4];
        const uint8_t cv = ct[(y0 + kk + 2) * CLX + x + 2];
        if (cv == 1) {
          T acc = 0;
          if (CROSS) {
            acc = A.S.cc * w[2][2];
            acc = fma(A.S.lx[0], w[2][0], acc);
            acc = fma(A.S.lx[1], w[2][1], acc);
            acc = fma(A.S.lx[3], w[2][3], acc);
            acc = fma(A.S.lx[4], w[2][4], acc);
            acc = fma(A.S.ly[0], w[0][2], acc);
            acc = fma(A.S.ly[1], w[1][2], acc);
            acc = fma(A.S.ly[3], w[3][2], acc);
            acc = fma(A.S.ly[4], w[4][2], acc);
            acc = fma(A.S.gy[0], D[0], acc);
            acc = fma(A.S.gy[1], D[1], acc);
            acc = fma(A.S.gy[3], D[3], acc);
            acc = fma(A.S.gy[4], D[4], acc);
          } else {
#pragma unroll
            for (int q = 0; q < 5; ++q)
#pragma unroll
              for (int b = 0; b < 5; ++b) {
                if (q != 2 && b != 2) continue;
                acc += A.S.w[q * 5 + b] * w[q][b];
              }
          }
          res[y0 + kk][x] = rt[(y0 + kk) * HX + x + 2] - acc;
        } else if (cv == 0) {
          res[y0 + kk][x] = (T)0;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
#pragma unroll
          for (int b = 0; b < 5; ++b) w[q][b] = w[q + 1][b];
          if (CROSS) D[q] = D[q + 1];
        }
      }
    }
    if (k + 1 < K) prefetch_tile_rows(A, n0, n1);
    __syncthreads();
    // 32 x 16 coarse cells, two per thread
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (cc[h] == 0) continue;
      const int c = threadIdx.x + h * 256;
      const int ci = c % (JX / 2), cj = c / (JX / 2);
      const long pc = (long)(cy0 / 2 + cj + 2) * A.pitchc + (cx0 / 2 + ci + 2);
      const T* v = vt + (2 * cj) * HX + 2 * ci + 2;
      const T v0 = v[0], v1 = v[1], v2 = v[HX], v3 = v[HX + 1];
      const T s = v0 * res[2 * cj][2 * ci] + v1 * res[2 * cj][2 * ci + 1] + v2 * res[2 * cj + 1][2 * ci] +
                  v3 * res[2 * cj + 1][2 * ci + 1];
      const T sv = v0 + v1 + v2 + v3;
      rcz[pc] = sv > (T)0 ? (T)4 * s / sv : (T)0;
      ucz[pc] = (T)0;
    }
    __syncthreads();      // res and stage sb are free
    if (threadIdx.x == 0 && k + 2 < K) {
      fence_proxy_async();
      issue(t + 2 * G, sb, 0);
    }
  }
}

}  // namespace dev
}  // namespace ccm
