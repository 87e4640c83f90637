// The small levels of a V-cycle (Alg. 2) in one launch of one thread-block cluster.
//
// Below a few hundred cells a side a level's smoothing sweep, restriction or prolongation
// costs a kernel launch and a grid drain, not bandwidth.  From level `first` down to the
// bottom level and back, this kernel runs every phase of Alg. 2 on one cluster of up to 16
// CTAs x 1024 threads, with the hardware cluster barrier between phases:
//   way down, per level: nu1 block-Jacobi sweeps (SMO-1 on the regular cells and the SMO-2
//     overlapping-block corrections of the irregular cells, both from the old iterate),
//     then residual + volume-weighted restriction and a zero coarse iterate;
//   bottom: the dense inverse of the bottom operator;
//   way up, per level: the first post-smoothing sweep reads u + P uc (the coarse correction
//     added to regular cells, Sec. 4.1) on the fly, then nu2 - 1 plain sweeps.
// The arithmetic is that of the multi-launch path cell by cell.  Every array that some CTA
// writes inside the launch is read with ld.global.cg (from L2), so that no CTA uses a stale
// L1 line of another CTA's writes; the cluster barrier's release/acquire orders the writes.
// No phase waits on anything but the cluster barrier, and every thread of every CTA passes
// the same sequence of barriers (no early exits).
#pragma once

#include "kernels.cuh"

namespace ccm {
namespace dev {

constexpr int MAXC = 8;           // levels one coarse launch covers
constexpr int COARSE_THREADS = 1024;

template <typename T>
struct CoarseLevel {
  int nx, ny, pitch, n2, nblk, nbc, W;
  const uint8_t* cls;
  const T* vol;
  T* u[2];
  T* r;
  const int32_t* irr_cell;
  const int32_t* rowmap;   // padded cell -> fitted row, -1 elsewhere
  const int32_t* colf;     // ELL columns (slot-major), sign bit set on regular columns
  const int32_t* par;      // per ELL slot: padded parent of a regular column, else -1
  const T* val;
  const int32_t* blk;      // per block: core rows [cs, ce), extended rows [es, ee)
  const int64_t* blk_off;
  const T* inv;            // per block: inverse rows [ext][core]
  const int32_t* bot_cell;
  const T* bot;            // bottom inverse, [col][row]
};

template <typename T>
struct CoarseParams {
  int nlev, nu1, nu2;
  int cur[MAXC];
  CoarseLevel<T> L[MAXC];
  Stencil<T> S;
};

__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ unsigned cluster_ctas() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}

// (h^2 L u) at a regular cell p from L2; with uc, u is read as u + P uc (regular cells only)
template <typename T, bool CROSS>
__device__ __forceinline__ T cl_stencil(const CoarseLevel<T>& L, const T* u, long p, int i, int j, const Stencil<T>& S,
                                        const T* uc, int pitchc, T& center) {
  T acc = 0;
#pragma unroll
  for (int dj = -2; dj <= 2; ++dj)
#pragma unroll
    for (int di = -2; di <= 2; ++di) {
      if (!CROSS && dj != 0 && di != 0) continue;
      const long q = p + (long)dj * L.pitch + di;
      T v = __ldcg(u + q);
      if (uc && L.cls[q] == 1) v += __ldcg(uc + (long)((j + dj) / 2 + 2) * pitchc + ((i + di) / 2 + 2));
      if (dj == 0 && di == 0) center = v;
      acc += S.w[(dj + 2) * 5 + di + 2] * v;
    }
  return acc;
}

// one block-Jacobi sweep u[1 - cur] <- u[cur] of a level: regular cells spread over all
// threads of the cluster, SMO-2 blocks over its CTAs
template <typename T, bool CROSS>
__device__ void cl_sweep(const CoarseLevel<T>& L, int cur, const Stencil<T>& S, const T* uc, int pitchc, T* sres,
                         T (*part)[33]) {
  const T* uin = L.u[cur];
  T* uout = L.u[1 - cur];
  const unsigned rank = cluster_rank(), nct = cluster_ctas();
  const int gtid = (int)(rank * blockDim.x + threadIdx.x), gsize = (int)(nct * blockDim.x);
  const int n = L.nx * L.ny;
  for (int idx = gtid; idx < n; idx += gsize) {
    const int i = idx % L.nx, j = idx / L.nx;
    const long p = (long)(j + 2) * L.pitch + (i + 2);
    if (L.cls[p] != 1) continue;
    T vp = 0;
    const T acc = cl_stencil<T, CROSS>(L, uin, p, i, j, S, uc, pitchc, vp);
    uout[p] = vp + S.omega_d * (__ldcg(L.r + p) - acc);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int b = (int)rank; b < L.nblk; b += (int)nct) {
    const int cs = L.blk[4 * b], ce = L.blk[4 * b + 1], es = L.blk[4 * b + 2], ee = L.blk[4 * b + 3];
    const int ne = ee - es, nc = ce - cs;
    for (int e = threadIdx.x; e < ne; e += blockDim.x) {
      const int row = es + e;
      T acc = 0;
#pragma unroll 15
      for (int k = 0; k < L.W; ++k) {
        const int f = L.colf[(long)k * L.n2 + row];
        const long q = f & 0x7fffffff;
        T v = __ldcg(uin + q);
        if (uc) {
          const int pq = L.par[(long)k * L.n2 + row];
          if (pq >= 0) v += __ldcg(uc + pq);
        }
        acc += L.val[(long)k * L.n2 + row] * v;
      }
      sres[e] = __ldcg(L.r + L.irr_cell[row]) - acc;
    }
    __syncthreads();
    const T* A = L.inv + L.blk_off[b];
    for (int cb = 0; cb < nc; cb += 32) {
      const int c = cb + lane;
      T acc = 0;
      if (c < nc)
        for (int e = warp; e < ne; e += nw) acc += A[(long)e * nc + c] * sres[e];
      part[warp][lane] = acc;
      __syncthreads();
      if (warp == 0 && c < nc) {
        T tot = 0;
        for (int w = 0; w < nw; ++w) tot += part[w][lane];
        const long q = L.irr_cell[cs + c];
        uout[q] = __ldcg(uin + q) + tot;
      }
      __syncthreads();
    }
  }
}

template <typename T, bool CROSS>
__global__ void __launch_bounds__(COARSE_THREADS, 1) k_coarse_cluster(CoarseParams<T> P) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* sres = reinterpret_cast<T*>(smem_raw);
  __shared__ T part[32][33];
  const unsigned rank = cluster_rank(), nct = cluster_ctas();
  const int gtid = (int)(rank * blockDim.x + threadIdx.x), gsize = (int)(nct * blockDim.x);
  int cur[MAXC];
#pragma unroll
  for (int m = 0; m < MAXC; ++m) cur[m] = P.cur[m];
  const int last = P.nlev - 1;
  for (int m = 0; m < last; ++m) {
    const CoarseLevel<T>& F = P.L[m];
    const CoarseLevel<T>& C = P.L[m + 1];
    for (int k = 0; k < P.nu1; ++k) {
      cl_sweep<T, CROSS>(F, cur[m], P.S, nullptr, 0, sres, part);
      cur[m] ^= 1;
      cluster_barrier();
    }
    // residual of every child (stencil or fitted row), volume-weighted restriction
    const T* u = F.u[cur[m]];
    T* ucz = C.u[cur[m + 1]];
    for (int idx = gtid; idx < C.nx * C.ny; idx += gsize) {
      const int I = idx % C.nx, J = idx / C.nx;
      const long pc = (long)(J + 2) * C.pitch + (I + 2);
      if (C.cls[pc] == 0) continue;
      const long f0 = (long)(2 * J + 2) * F.pitch + (2 * I + 2);
      T s = 0, sv = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const long q = f0 + (k >> 1) * (long)F.pitch + (k & 1);
        const uint8_t c = F.cls[q];
        if (c == 0) continue;
        T Lu = 0;
        if (c == 1) {
          T center;
          Lu = cl_stencil<T, CROSS>(F, u, q, 2 * I + (k & 1), 2 * J + (k >> 1), P.S, nullptr, 0, center);
        } else {
          const int row = F.rowmap[q];
#pragma unroll 15
          for (int t = 0; t < F.W; ++t)
            Lu += F.val[(long)t * F.n2 + row] * __ldcg(u + (F.colf[(long)t * F.n2 + row] & 0x7fffffff));
        }
        const T v = F.vol[q];
        s += v * (__ldcg(F.r + q) - Lu);
        sv += v;
      }
      C.r[pc] = sv > (T)0 ? (T)4 * s / sv : (T)0;
      ucz[pc] = (T)0;
    }
    cluster_barrier();
  }
  {
    // bottom: u = inv(L_bottom) r; every CTA stages r, 32-row groups over the CTAs,
    // the columns over the warps of a CTA
    const CoarseLevel<T>& B = P.L[last];
    T* u = B.u[cur[last]];
    for (int c = threadIdx.x; c < B.nbc; c += blockDim.x) sres[c] = __ldcg(B.r + B.bot_cell[c]);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int g = (int)rank; g * 32 < B.nbc; g += (int)nct) {
      const int k = g * 32 + lane;
      T acc = 0;
      if (k < B.nbc)
        for (int c = warp; c < B.nbc; c += nw) acc += B.bot[(long)c * B.nbc + k] * sres[c];
      part[warp][lane] = acc;
      __syncthreads();
      if (warp == 0 && k < B.nbc) {
        T tot = 0;
        for (int w = 0; w < nw; ++w) tot += part[w][lane];
        u[B.bot_cell[k]] = tot;
      }
      __syncthreads();
    }
    cluster_barrier();
  }
  for (int m = last - 1; m >= 0; --m) {
    const CoarseLevel<T>& F = P.L[m];
    const CoarseLevel<T>& C = P.L[m + 1];
    const T* uc = C.u[cur[m + 1]];
    if (P.nu2 == 0) {
      T* u = F.u[cur[m]];
      for (int idx = gtid; idx < F.nx * F.ny; idx += gsize) {
        const int i = idx % F.nx, j = idx / F.nx;
        const long p = (long)(j + 2) * F.pitch + (i + 2);
        if (F.cls[p] == 1) u[p] = __ldcg(u + p) + __ldcg(uc + (long)(j / 2 + 2) * C.pitch + (i / 2 + 2));
      }
      cluster_barrier();
      continue;
    }
    for (int k = 0; k < P.nu2; ++k) {
      cl_sweep<T, CROSS>(F, cur[m], P.S, k == 0 ? uc : nullptr, C.pitch, sres, part);
      cur[m] ^= 1;
      cluster_barrier();
    }
  }
}

}  // namespace dev
}  // namespace ccm
