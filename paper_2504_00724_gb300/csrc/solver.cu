// Device side of the solver: level arrays, the V-cycle of Alg. 2 on the stream, the FP64
// outer iteration (plain FP64 cycles, or FP32 cycles inside FP64 iterative refinement),
// and the C ABI of include/ccm.h.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include "hierarchy.h"
#include "kernels.cuh"
#include "coarse.cuh"
#include "smooth.cuh"
#include "outer.cuh"
#include "group.cuh"
#include "krylov.cuh"

using namespace ccm;

namespace {

struct DevLevel {
  int nx = 0, ny = 0, pitch = 0, rows = 0, ntiles = 0, n2 = 0, W = 15, nblk = 0, nbc = 0, ncolT = 0;
  long npad = 0;
  double h = 0;
  int max_ext = 0, max_core = 0;
  int32_t* tiles = nullptr;
  int ntiles64 = 0;
  int32_t* tiles64 = nullptr;
  int ntiles64r = 0;            // fine 64 x 32 tiles that restriction to level m + 1 visits
  int32_t* tiles64r = nullptr;
  bool stage_blocks = false;    // SMO-2 block inverses fit in shared memory (bulk-staged kernel)
  bool tma = false;             // TMA-staged SMO-1 on this level
  CUtensorMap tm64[2], tm32[2]; // 68 x 36 boxes over the u buffers
  CUtensorMap tmcls;            // 80 x 36 box over the class bytes
  CUtensorMap tmuc64[2], tmuc32[2];  // 36 x 18 boxes over level m + 1's u buffers
  bool tma_pro = false;         // the maps above exist: prolongation fuses into the sweep
  CUtensorMap tmr64, tmr32;     // 68 x 32 boxes over r
  bool smooth_ok[2] = {false, false};  // persistent sweep (k_smooth) usable, [0] FP64, [1] FP32
  uint32_t smooth_stage[2] = {0, 0};
  size_t smooth_smem[2] = {0, 0};
  int smooth_grid[2] = {0, 0};
  int smooth_cap[2] = {0, 0};   // resident CTAs of the persistent sweep over the whole GPU
  CUtensorMap tmv64, tmv32;     // 68 x 32 boxes over the cell volumes
  bool restrict_ok[2] = {false, false};  // persistent restriction (k_restrict_p), [0] FP64, [1] FP32
  uint32_t restrict_stage[2] = {0, 0};
  int restrict_grid[2] = {0, 0};
  int restrict_cap[2] = {0, 0};
  int32_t* rr_off = nullptr;    // per restriction tile: its irregular rows [rr_off[t], rr_off[t + 1])
  int32_t* rr = nullptr;        // (row, y * 64 + x in the tile) pairs
  // the same rows packed in restriction-tile order for k_restrict_p: (cell, y * 64 + x) pairs
  // and the fitted rows' columns and coefficients [W][nrr], so that one tile's rows are
  // contiguous (coalesced, and prefetched while the tile before is restricted)
  int nrr = 0;
  int32_t *rq = nullptr, *rq_col = nullptr;
  double* rq_val64 = nullptr;
  float* rq_val32 = nullptr;
  uint8_t* cls = nullptr;
  double* vol64 = nullptr;
  float* vol32 = nullptr;
  int32_t *irr_cell = nullptr, *ell_col = nullptr, *ell_colf = nullptr, *seg = nullptr, *rowmap = nullptr;
  int32_t* ell_par = nullptr;   // per ELL slot: padded parent of a regular column (level m + 1), else -1
  double *ell64 = nullptr, *nb = nullptr;
  float* ell32 = nullptr;
  int32_t *order = nullptr, *blk = nullptr;
  int64_t* blk_off = nullptr;
  double* inv64 = nullptr;
  float* inv32 = nullptr;
  int32_t* bot_cell = nullptr;
  double* bot64 = nullptr;
  float* bot32 = nullptr;
  int32_t *tr_ptr = nullptr, *tr_cell = nullptr, *tr_row = nullptr;
  double* tr_val = nullptr;
  // work arrays (padded), FP64 and FP32 sets
  double *u64[2] = {nullptr, nullptr}, *r64 = nullptr, *t64 = nullptr, *res64 = nullptr;
  float *u32[2] = {nullptr, nullptr}, *r32 = nullptr, *t32 = nullptr, *res32 = nullptr;
  int cur64 = 0, cur32 = 0;
};

template <typename T> T* U(DevLevel& L);
template <> double* U<double>(DevLevel& L) { return L.u64[L.cur64]; }
template <> float* U<float>(DevLevel& L) { return L.u32[L.cur32]; }
template <typename T> const CUtensorMap& TmU(const DevLevel& L);
template <> const CUtensorMap& TmU<double>(const DevLevel& L) { return L.tm64[L.cur64]; }
template <> const CUtensorMap& TmU<float>(const DevLevel& L) { return L.tm32[L.cur32]; }
template <typename T> T* Uother(DevLevel& L);
template <> double* Uother<double>(DevLevel& L) { return L.u64[1 - L.cur64]; }
template <> float* Uother<float>(DevLevel& L) { return L.u32[1 - L.cur32]; }
template <typename T> void flip(DevLevel& L);
template <> void flip<double>(DevLevel& L) { L.cur64 = 1 - L.cur64; }
template <> void flip<float>(DevLevel& L) { L.cur32 = 1 - L.cur32; }
template <typename T> T* R(DevLevel& L);
template <> double* R<double>(DevLevel& L) { return L.r64; }
template <> float* R<float>(DevLevel& L) { return L.r32; }
template <typename T> T* Tmp(DevLevel& L);
template <> double* Tmp<double>(DevLevel& L) { return L.t64; }
template <> float* Tmp<float>(DevLevel& L) { return L.t32; }
template <typename T> T* Res(DevLevel& L);
template <> double* Res<double>(DevLevel& L) { return L.res64; }
template <> float* Res<float>(DevLevel& L) { return L.res32; }
template <typename T> const T* Ell(const DevLevel& L);
template <> const double* Ell<double>(const DevLevel& L) { return L.ell64; }
template <> const float* Ell<float>(const DevLevel& L) { return L.ell32; }
template <typename T> const T* RqVal(const DevLevel& L);
template <> const double* RqVal<double>(const DevLevel& L) { return L.rq_val64; }
template <> const float* RqVal<float>(const DevLevel& L) { return L.rq_val32; }
template <typename T> const T* Inv(const DevLevel& L);
template <> const double* Inv<double>(const DevLevel& L) { return L.inv64; }
template <> const float* Inv<float>(const DevLevel& L) { return L.inv32; }
template <typename T> const T* Vol(const DevLevel& L);
template <> const double* Vol<double>(const DevLevel& L) { return L.vol64; }
template <> const float* Vol<float>(const DevLevel& L) { return L.vol32; }
template <typename T> const T* Bot(const DevLevel& L);
template <> const double* Bot<double>(const DevLevel& L) { return L.bot64; }
template <> const float* Bot<float>(const DevLevel& L) { return L.bot32; }

struct Arena {
  std::vector<void*> blocks;
  std::vector<long> sizes;
  long bytes = 0;
  cudaError_t err = cudaSuccess;
  template <typename T>
  T* alloc(long n, bool zero = true) {
    if (n <= 0 || err != cudaSuccess) return nullptr;
    void* p = nullptr;
    err = cudaMalloc(&p, n * sizeof(T));
    if (err != cudaSuccess) return nullptr;
    if (zero) err = cudaMemset(p, 0, n * sizeof(T));
    blocks.push_back(p);
    sizes.push_back(n * (long)sizeof(T));
    bytes += n * (long)sizeof(T);
    return (T*)p;
  }
  // give one earlier allocation back (nullptr: nothing)
  void free(void* p) {
    if (!p) return;
    for (size_t k = 0; k < blocks.size(); ++k)
      if (blocks[k] == p) {
        cudaFree(p);
        bytes -= sizes[k];
        blocks.erase(blocks.begin() + k);
        sizes.erase(sizes.begin() + k);
        return;
      }
  }
  template <typename T>
  T* upload(const std::vector<T>& v) {
    T* p = alloc<T>((long)v.size(), false);
    if (p && err == cudaSuccess) err = cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
    return p;
  }
  void release() {
    for (void* p : blocks) cudaFree(p);
    blocks.clear();
    sizes.clear();
  }
};

}  // namespace

struct ccm_handle {
  ccm_params par{};
  double a = 0, b = 0, c = 0;
  bool cross = false;
  Hierarchy H;
  std::vector<DevLevel> L;
  Arena arena;
  dev::Stencil<double> S64{};
  dev::Stencil<float> S32{};
  int* derr = nullptr;         // device error word (bounded waits that ran out)
  int* herr = nullptr;         // pinned copy
  double* rhat = nullptr;      // level-0 padded FP64 right-hand side (h^2-scaled)
  double* uhat = nullptr;      // level-0 padded FP64 solution
  bool fused_outer = false;    // mixed form: TMA-tiled FP64 residual writing r32 and the norm
  int B = 1;                   // right-hand sides the FP32 work arrays and level-0 FP64 arrays hold
  int bmax = 1;                // right-hand sides one graph replay advances (B where batching applies)
  int nb = 1;                  // right-hand sides of the launches being issued (<= bmax)
  CUtensorMap tm_uhat, tm_rhat;  // 68 x 36 box over uhat, 68 x 32 box over rhat
  dev::SepStencil sep{};       // the regular stencil in factored form
  dev::FFStencil ffs{};        // its three coefficients as FP32 pairs (float-float residual)
  unsigned long long* dnorm = nullptr;
  unsigned long long* hnorm = nullptr;   // pinned
  ccm_info info{};
  int device = 0;
  // kernel-class profiling (ccm_profile): event pairs around the chosen class of launches
  int prof_class = 0;
  std::vector<cudaEvent_t> prof_ev;   // stream-mode pairs (read at ccm_profile_read)
  int prof_used = 0;
  std::vector<cudaEvent_t> gprof_ev;  // pairs baked into the iteration graphs
  double prof_ms = 0;                 // accumulated from graph replays
  long long prof_n = 0;
  int coarse_first = 1 << 30;  // first level whose part of the V-cycle runs as one cluster launch
  int coarse_ctas = 0;         // CTAs of that cluster (16, else 8)
  size_t coarse_smem = 0;      // its dynamic shared memory (SMO-2 extended-row residuals)
  bool persistent = true;      // block-Jacobi sweeps of TMA levels as one persistent launch
  int launch_cap = 0;          // > 0: at most this many CTAs per right-hand side in the persistent kernels
  // GMRES(kry_m) correction of the mixed outer iteration (0: plain iterative refinement)
  int kry_m = 0;
  float* kv[dev::KRY_MAXM + 1] = {};   // Krylov basis v_0 .. v_m (padded level-0 FP32 arrays)
  float* kz[dev::KRY_MAXM] = {};       // preconditioned vectors z_j = M v_j
  dev::KryScalars* ks = nullptr;
  ccm_handle* adj = nullptr;   // the transposed operators' hierarchy (built by ccm_solve_T)
  // one CUDA graph per outer iteration and precision (captured on first use, on a private
  // stream: the legacy default stream cannot be captured)
  cudaStream_t cap_stream = nullptr;
  cudaStream_t side = nullptr;          // second stream: SMO-2 blocks beside the regular sweep
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool capturing = false;
  // one-launch requests to the next persistent FP32 sweep (set while a V-cycle is issued,
  // cleared when used): zero_u_next, its old iterate is 0 (not read; a level's first sweep);
  // fold_next (level 0), it also adds its new values to u_hat (the outer iteration's update).
  // fold_last marks the last inner cycle; folded reports that a sweep took the update.
  bool zero_u_next = false, fold_next = false, fold_last = false, folded = false;
  long long cap_launches = 0;
  struct Graph {
    cudaGraphExec_t exec = nullptr;
    long long launches = 0;
    std::vector<int> prof_pairs;      // indices into gprof_ev (pairs at 2k, 2k + 1)
    double* u0 = nullptr;             // the level-0 FP64 iterate the graph updates
    int nb = 1;                       // right-hand sides its launches cover
  } graph[2];
};

namespace {

inline int ceil_div(long a, long b) { return (int)((a + b - 1) / b); }

// CTAs per right-hand side of a persistent launch: every item gets its own CTA up to the
// resident capacity shared by the nb right-hand sides, and at most the handle's launch cap
inline int persistent_ctas(int items_grid, int cap, int nb, int launch_cap) {
  int g = std::min(items_grid, std::max(1, ceil_div(cap, nb)));
  if (launch_cap > 0) g = std::min(g, launch_cap);
  return std::max(1, g);
}

std::atomic<long long> g_launches{0};
// every kernel launch of the library goes through KL so that launches can be counted
#define KL(...) (g_launches.fetch_add(1, std::memory_order_relaxed), __VA_ARGS__)

// event pair around the launches of the profiled class
struct ProfScope {
  ccm_handle* H;
  cudaStream_t s;
  bool on;
  int gidx = -1;
  ProfScope(ccm_handle* H_, int cls, cudaStream_t s_) : H(H_), s(s_), on(cls != 0 && H_->prof_class == cls) {
    if (!on) return;
    if (H->capturing) {
      cudaEvent_t a, b;
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      gidx = (int)H->gprof_ev.size();
      H->gprof_ev.push_back(a);
      H->gprof_ev.push_back(b);
      cudaEventRecordWithFlags(a, s, cudaEventRecordExternal);   // a real record node in the graph
      return;
    }
    if (H->prof_used + 2 > (int)H->prof_ev.size()) {
      for (int k = 0; k < 512; ++k) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        H->prof_ev.push_back(e);
      }
    }
    cudaEventRecord(H->prof_ev[H->prof_used], s);
  }
  ~ProfScope() {
    if (!on) return;
    if (gidx >= 0) {
      cudaEventRecordWithFlags(H->gprof_ev[gidx + 1], s, cudaEventRecordExternal);
      return;
    }
    cudaEventRecord(H->prof_ev[H->prof_used + 1], s);
    H->prof_used += 2;
  }
};


#define CCM_CUDA(call)                                  \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return CCM_ECUDA;            \
  } while (0)

// launches of this thread carry the programmatic-serialization attribute (cleared while a
// graph is captured for a runtime that does not take programmatic edges inside conditional
// bodies)
thread_local bool t_pdl = true;

// kernel launch with programmatic stream serialization (the kernel may start while the
// previous kernel of the stream drains; it waits for it inside, see pdl_enter)
template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*k)(KArgs...), dim3 g, dim3 b, size_t smem, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg{};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.gridDim = g;
  cfg.blockDim = b;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = t_pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, args...);
}

// ---------------------------------------------------------------- level operations

template <typename T>
void launch_regular(ccm_handle* H, DevLevel& L, const T* u, const T* r, T* out, bool resid, cudaStream_t s);

template <typename T>
const dev::Stencil<T>& stencil(ccm_handle* H);
template <> const dev::Stencil<double>& stencil<double>(ccm_handle* H) { return H->S64; }
template <> const dev::Stencil<float>& stencil<float>(ccm_handle* H) { return H->S32; }

template <typename T>
void launch_regular(ccm_handle* H, DevLevel& L, const T* u, const T* r, T* out, bool resid, cudaStream_t s) {
  if (L.ntiles == 0) return;
  dim3 blk(dev::TX, dev::TY);
  const auto& S = stencil<T>(H);
  if (H->cross) {
    if (resid) KL(launch_k(dev::k_regular<T, true, true>, L.ntiles, blk, 0, s, L.tiles, L.cls, L.nx, L.ny, L.pitch, u, r, out, S));
    else KL(launch_k(dev::k_regular<T, true, false>, L.ntiles, blk, 0, s, L.tiles, L.cls, L.nx, L.ny, L.pitch, u, r, out, S));
  } else {
    if (resid) KL(launch_k(dev::k_regular<T, false, true>, L.ntiles, blk, 0, s, L.tiles, L.cls, L.nx, L.ny, L.pitch, u, r, out, S));
    else KL(launch_k(dev::k_regular<T, false, false>, L.ntiles, blk, 0, s, L.tiles, L.cls, L.nx, L.ny, L.pitch, u, r, out, S));
  }
}

// out = r - L u on every non-empty cell of the level (grid layout)
template <typename T>
void residual(ccm_handle* H, DevLevel& L, const T* u, const T* r, T* out, cudaStream_t s) {
  launch_regular<T>(H, L, u, r, out, true, s);
  if (L.n2)
    KL(launch_k(dev::k_rows<T, T, true, true>, ceil_div(L.n2, 128), 128, 0, s, L.n2, L.W, L.irr_cell, L.ell_col, Ell<T>(L), u, r, out,
                                                                      nullptr, nullptr, nullptr));
}

// one smoother step: SMO-1 on the regular cells, then SMO-2 on the irregular cells.
// uc != nullptr fuses the prolongation u += P uc into the SMO-1 sweep (regular cells).
template <typename T>
void prolong_from(ccm_handle* H, DevLevel& F, DevLevel& C, cudaStream_t s);

template <typename T> const CUtensorMap& TmUc(const DevLevel& F, const DevLevel& C);
template <> const CUtensorMap& TmUc<double>(const DevLevel& F, const DevLevel& C) { return F.tmuc64[C.cur64]; }
template <> const CUtensorMap& TmUc<float>(const DevLevel& F, const DevLevel& C) { return F.tmuc32[C.cur32]; }

// block-Jacobi form: SMO-1 and SMO-2 both from the old iterate, one launch (plus the SMO-2
// blocks on a parallel branch where their inverses are staged).  C != null: the first
// post-smoothing sweep, which reads u + P uc with uc the iterate of level C.
template <typename T> const CUtensorMap& TmR(const DevLevel& L);
template <> const CUtensorMap& TmR<double>(const DevLevel& L) { return L.tmr64; }
template <> const CUtensorMap& TmR<float>(const DevLevel& L) { return L.tmr32; }

// the persistent sweep (k_smooth): SMO-2 block items and TMA tile items in one launch
template <typename T>
void sweep_persistent(ccm_handle* H, DevLevel& L, cudaStream_t s, DevLevel* C) {
  const int k = sizeof(T) == 8 ? 0 : 1;
  dev::SmoothArgs<T> A{};
  dev::SweepArgs<T>& a = A.a;
  a.tiles = L.tiles64;
  a.ntiles = L.ntiles64;
  a.nblk = L.nblk;
  a.chunks = 1;
  a.cls = L.cls;
  a.nx = L.nx;
  a.ny = L.ny;
  a.pitch = L.pitch;
  a.n2 = L.n2;
  a.W = L.W;
  a.r = R<T>(L);
  a.u_old = U<T>(L);
  a.u_new = Uother<T>(L);
  a.S = stencil<T>(H);
  a.blk = L.blk;
  a.blk_off = L.blk_off;
  a.inv = Inv<T>(L);
  a.cell = L.irr_cell;
  a.col = L.ell_col;
  a.val = Ell<T>(L);
  a.err = H->derr;
  a.par = L.ell_par;
  a.uc = C ? U<T>(*C) : nullptr;
  A.nbi = L.nblk;
  A.nitems = L.nblk + L.ntiles64;
  A.stage = L.smooth_stage[k];
  A.max_ext = std::max(1, L.max_ext);
  const bool l0f = &L == &H->L[0] && sizeof(T) == 4;
  a.zero_u = sizeof(T) == 4 && !C && H->zero_u_next ? 1 : 0;
  a.uhat = l0f && H->fold_next ? H->uhat : nullptr;
  if (a.uhat) H->folded = true;
  H->zero_u_next = H->fold_next = false;
  const bool l0 = &L == &H->L[0];
  ProfScope ps(H, !l0 ? 0 : C ? (sizeof(T) == 4 ? CCM_PROF_PROLONG_SMO1_FP32 : 0)
                              : (sizeof(T) == 4 ? CCM_PROF_SMO1_FP32 : CCM_PROF_SMO1_FP64), s);
  const CUtensorMap& tm = TmU<T>(L);
  const CUtensorMap& tr = TmR<T>(L);
  a.bs = L.npad;
  a.bsc = C ? C->npad : 0;
  // with a batch, fewer CTAs per right-hand side so that the whole launch stays resident
  const dim3 grid(persistent_ctas(L.smooth_grid[k], L.smooth_cap[k], H->nb, H->launch_cap), H->nb);
  const size_t smem = L.smooth_smem[k];
  if (C) {
    const CUtensorMap& tu = TmUc<T>(L, *C);
    if (H->cross) KL(launch_k(dev::k_smooth<T, true, true>, grid, 256, smem, s, tm, tr, L.tmcls, tu, A));
    else KL(launch_k(dev::k_smooth<T, false, true>, grid, 256, smem, s, tm, tr, L.tmcls, tu, A));
  } else {
    if (H->cross) KL(launch_k(dev::k_smooth<T, true, false>, grid, 256, smem, s, tm, tr, L.tmcls, tm, A));
    else KL(launch_k(dev::k_smooth<T, false, false>, grid, 256, smem, s, tm, tr, L.tmcls, tm, A));
  }
}

template <typename T>
void sweep_one_launch(ccm_handle* H, DevLevel& L, cudaStream_t s, DevLevel* C = nullptr) {
  if (L.smooth_ok[sizeof(T) == 8 ? 0 : 1] && H->persistent) {
    if (C && !L.tma_pro) {
      prolong_from<T>(H, L, *C, s);
      C = nullptr;
    }
    sweep_persistent<T>(H, L, s, C);
    return;
  }
  const bool staged = L.tma && (L.nblk == 0 || L.stage_blocks);
  if (C && !(staged && L.tma_pro)) {
    prolong_from<T>(H, L, *C, s);
    C = nullptr;
  }
  dev::SweepArgs<T> a{};
  const bool tma = L.tma;
  a.tiles = tma ? L.tiles64 : L.tiles;
  a.ntiles = tma ? L.ntiles64 : L.ntiles;
  a.nblk = L.nblk;
  a.rows_per_cta = L.nblk >= 16 ? std::max(1, L.max_core) : 64;
  a.chunks = L.nblk ? ceil_div(std::max(1, L.max_core), a.rows_per_cta) : 0;
  a.cls = L.cls;
  a.nx = L.nx;
  a.ny = L.ny;
  a.pitch = L.pitch;
  a.n2 = L.n2;
  a.W = L.W;
  a.r = R<T>(L);
  a.u_old = U<T>(L);
  a.u_new = Uother<T>(L);
  a.S = stencil<T>(H);
  a.blk = L.blk;
  a.blk_off = L.blk_off;
  a.inv = Inv<T>(L);
  a.cell = L.irr_cell;
  a.col = L.ell_col;
  a.val = Ell<T>(L);
  a.err = H->derr;
  a.par = L.ell_par;
  a.uc = C ? U<T>(*C) : nullptr;
  a.bs = L.npad;
  a.bsc = C ? C->npad : 0;
  const bool l0 = &L == &H->L[0];
  ProfScope ps(H, !l0 ? 0 : C ? (sizeof(T) == 4 ? CCM_PROF_PROLONG_SMO1_FP32 : 0)
                              : (sizeof(T) == 4 ? CCM_PROF_SMO1_FP32 : CCM_PROF_SMO1_FP64), s);
  if (L.stage_blocks && a.nblk) {
    // SMO-2 blocks on the side stream, regular cells here; join before the next phase
    dev::SweepArgs<T> b = a;
    b.ntiles = 0;
    b.tiles = nullptr;
    a.nblk = 0;
    cudaEventRecord(H->ev_fork, s);
    cudaStreamWaitEvent(H->side, H->ev_fork, 0);
    const size_t bsm = (((size_t)L.max_ext * L.max_core * sizeof(T) + 15) & ~(size_t)15) + L.max_ext * sizeof(T);
    KL(dev::k_blocks<T><<<dim3(b.nblk * b.chunks, H->nb), 256, bsm, H->side>>>(b));
    cudaEventRecord(H->ev_join, H->side);
  }
  const CUtensorMap& tm = TmU<T>(L);
  if (staged && a.ntiles) {
    if (C) {
      const CUtensorMap& tu = TmUc<T>(L, *C);
      if (H->cross) KL(launch_k(dev::k_sweep_tma<T, true, true>, a.ntiles, 256, 0, s, tm, L.tmcls, tu, a));
      else KL(launch_k(dev::k_sweep_tma<T, false, true>, a.ntiles, 256, 0, s, tm, L.tmcls, tu, a));
    } else {
      if (H->cross) KL(launch_k(dev::k_sweep_tma<T, true, false>, a.ntiles, 256, 0, s, tm, tm, tm, a));
      else KL(launch_k(dev::k_sweep_tma<T, false, false>, a.ntiles, 256, 0, s, tm, tm, tm, a));
    }
  } else {
    const int grid = a.ntiles + a.nblk * a.chunks;
    const size_t smem = (size_t)std::max(1, L.max_ext) * sizeof(T);
    if (grid > 0) {
      if (tma) {
        if (H->cross) KL(launch_k(dev::k_sweep<T, true, true>, grid, 256, smem, s, tm, a));
        else KL(launch_k(dev::k_sweep<T, false, true>, grid, 256, smem, s, tm, a));
      } else {
        if (H->cross) KL(launch_k(dev::k_sweep<T, true, false>, dim3(grid, H->nb), 256, smem, s, tm, a));
        else KL(launch_k(dev::k_sweep<T, false, false>, dim3(grid, H->nb), 256, smem, s, tm, a));
      }
    }
  }
  if (L.stage_blocks && L.nblk) cudaStreamWaitEvent(s, H->ev_join, 0);
}

template <typename T>
void smooth_step(ccm_handle* H, DevLevel& L, cudaStream_t s, const T* uc = nullptr, int pitchc = 0) {
  if (H->par.smoother == 1 && H->par.ras_passes <= 1) {
    sweep_one_launch<T>(H, L, s, uc ? &H->L[&L - &H->L[0] + 1] : nullptr);
    flip<T>(L);
    return;
  }
  T* uin = U<T>(L);
  T* uout = Uother<T>(L);
  const T* r = R<T>(L);
  if (L.ntiles) {
    dim3 blk(dev::TX, dev::TY);
    const auto& S = stencil<T>(H);
    const bool l0 = &L == &H->L[0];
    ProfScope ps(H, !l0 ? 0 : uc ? (sizeof(T) == 4 ? CCM_PROF_PROLONG_SMO1_FP32 : 0)
                              : (sizeof(T) == 4 ? CCM_PROF_SMO1_FP32 : CCM_PROF_SMO1_FP64), s);
    if (!uc && L.tma) {
      if (H->cross) KL(dev::k_jacobi_tma<T, true><<<L.ntiles64, 256, 0, s>>>(TmU<T>(L), L.tiles64, L.cls, L.nx, L.ny, L.pitch, r, uout, S, H->derr));
      else KL(dev::k_jacobi_tma<T, false><<<L.ntiles64, 256, 0, s>>>(TmU<T>(L), L.tiles64, L.cls, L.nx, L.ny, L.pitch, r, uout, S, H->derr));
    } else if (uc) {
      if (H->cross) KL(dev::k_jacobi2<T, true, true><<<L.ntiles, blk, 0, s>>>(L.tiles, L.cls, L.nx, L.ny, L.pitch, pitchc, uin, uc, uout, r, S));
      else KL(dev::k_jacobi2<T, false, true><<<L.ntiles, blk, 0, s>>>(L.tiles, L.cls, L.nx, L.ny, L.pitch, pitchc, uin, uc, uout, r, S));
    } else {
      if (H->cross) KL(dev::k_jacobi2<T, true, false><<<L.ntiles, blk, 0, s>>>(L.tiles, L.cls, L.nx, L.ny, L.pitch, 0, uin, nullptr, uout, r, S));
      else KL(dev::k_jacobi2<T, false, false><<<L.ntiles, blk, 0, s>>>(L.tiles, L.cls, L.nx, L.ny, L.pitch, 0, uin, nullptr, uout, r, S));
    }
  }
  if (L.n2) {
    ProfScope ps(H, (&L == &H->L[0] && sizeof(T) == 4) ? CCM_PROF_SMO2_FP32 : 0, s);
    // many blocks: one CTA each; one big exact block: split its core rows over CTAs
    const int rpc = L.nblk >= 16 ? L.max_core : 64;
    dim3 grd(L.nblk, ceil_div(L.max_core, rpc));
    KL(dev::k_block_fused<T><<<grd, 256, L.max_ext * sizeof(T), s>>>(L.blk, L.blk_off, Inv<T>(L), L.n2, L.W, L.irr_cell,
                                                                  L.ell_colf, Ell<T>(L), r, uin, uout, rpc));
  }
  flip<T>(L);
  T* u = U<T>(L);
  for (int pass = 1; pass < H->par.ras_passes && L.n2; ++pass) {
    KL(launch_k(dev::k_rows<T, T, true, false>, ceil_div(L.n2, 128), 128, 0, s, L.n2, L.W, L.irr_cell, L.ell_col, Ell<T>(L), u, r,
                                                                       Res<T>(L), nullptr, nullptr, nullptr));
    dim3 grd(L.nblk, ceil_div(L.max_core, 32));
    KL(dev::k_block_solve<T><<<grd, 128, L.max_ext * sizeof(T), s>>>(L.order, L.blk, L.blk_off, Inv<T>(L), Res<T>(L),
                                                                  L.irr_cell, u));
  }
}

// residual, restriction and zeroing of the coarse iterate
template <typename T>
void restrict_to(ccm_handle* H, DevLevel& F, DevLevel& C, cudaStream_t s) {
  ProfScope ps(H, (&F == &H->L[0] && sizeof(T) == 4) ? CCM_PROF_RESTRICT_FP32 : 0, s);
  const int kk = sizeof(T) == 8 ? 0 : 1;
  if (H->par.smoother == 1 && F.tma && F.ntiles64r && F.restrict_ok[kk] && H->persistent) {
    dev::RestrictArgs<T> A{};
    A.tiles = F.tiles64r;
    A.ntiles = F.ntiles64r;
    A.nxf = F.nx;
    A.nyf = F.ny;
    A.pitchf = F.pitch;
    A.rr_off = F.rr_off;
    A.rr = F.rr;
    A.nrr = F.nrr;
    A.rq = F.rq;
    A.rq_col = F.rq_col;
    A.rq_val = RqVal<T>(F);
    A.n2 = F.n2;
    A.W = F.W;
    A.irr_cell = F.irr_cell;
    A.col = F.ell_col;
    A.val = Ell<T>(F);
    A.u = U<T>(F);
    A.r = R<T>(F);
    A.nxc = C.nx;
    A.nyc = C.ny;
    A.pitchc = C.pitch;
    A.clsc = C.cls;
    A.rc = R<T>(C);
    A.uc = U<T>(C);
    A.S = stencil<T>(H);
    A.err = H->derr;
    A.stage = F.restrict_stage[kk];
    A.bs = F.npad;
    A.bsc = C.npad;
    const CUtensorMap& tv = kk == 0 ? F.tmv64 : F.tmv32;
    const size_t smem = 2 * (size_t)A.stage;
    const dim3 rgrid(persistent_ctas(F.restrict_grid[kk], F.restrict_cap[kk], H->nb, H->launch_cap), H->nb);
    if (H->cross)
      KL(launch_k(dev::k_restrict_p<T, true>, rgrid, 256, smem, s, TmU<T>(F), TmR<T>(F), F.tmcls, tv, A));
    else
      KL(launch_k(dev::k_restrict_p<T, false>, rgrid, 256, smem, s, TmU<T>(F), TmR<T>(F), F.tmcls, tv, A));
    return;
  }
  if (H->par.smoother == 1 && F.tma && F.ntiles64r) {
    const auto& S = stencil<T>(H);
    if (H->cross)
      KL(launch_k(dev::k_restrict_tma<T, true>, F.ntiles64r, 256, 0, s, TmU<T>(F), F.tiles64r, F.nx, F.ny, F.pitch, F.cls, Vol<T>(F),
                                                         F.rr_off, F.rr, F.n2, F.W, F.irr_cell, F.ell_col, Ell<T>(F),
                                                         U<T>(F), R<T>(F), C.nx, C.ny, C.pitch, C.cls, R<T>(C), U<T>(C), S,
                                                         H->derr));
    else
      KL(launch_k(dev::k_restrict_tma<T, false>, F.ntiles64r, 256, 0, s, TmU<T>(F), F.tiles64r, F.nx, F.ny, F.pitch, F.cls, Vol<T>(F),
                                                         F.rr_off, F.rr, F.n2, F.W, F.irr_cell, F.ell_col, Ell<T>(F),
                                                         U<T>(F), R<T>(F), C.nx, C.ny, C.pitch, C.cls, R<T>(C), U<T>(C), S,
                                                         H->derr));
    return;
  }
  if (H->par.smoother == 1) {
    dim3 blk(32, 8), grd(ceil_div(C.nx, 32), ceil_div(C.ny, 8), H->nb);
    const auto& S = stencil<T>(H);
    if (H->cross)
      KL(launch_k(dev::k_restrict_rows<T, true>, grd, blk, 0, s, C.nx, C.ny, C.pitch, F.pitch, C.cls, F.cls, Vol<T>(F), F.rowmap,
                  F.n2, F.W, F.ell_col, Ell<T>(F), U<T>(F), R<T>(F), R<T>(C), U<T>(C), S, F.npad, C.npad));
    else
      KL(launch_k(dev::k_restrict_rows<T, false>, grd, blk, 0, s, C.nx, C.ny, C.pitch, F.pitch, C.cls, F.cls, Vol<T>(F), F.rowmap,
                  F.n2, F.W, F.ell_col, Ell<T>(F), U<T>(F), R<T>(F), R<T>(C), U<T>(C), S, F.npad, C.npad));
    return;
  }
  if (F.n2)
    KL(launch_k(dev::k_rows<T, T, true, true>, ceil_div(F.n2, 128), 128, 0, s, F.n2, F.W, F.irr_cell, F.ell_col, Ell<T>(F), U<T>(F),
                                                                      R<T>(F), Tmp<T>(F), nullptr, nullptr, nullptr));
  dim3 blk(32, 8), grd(ceil_div(C.nx, 32), ceil_div(C.ny, 8));
  const auto& S = stencil<T>(H);
  if (H->cross)
    KL(dev::k_restrict_fused<T, true><<<grd, blk, 0, s>>>(C.nx, C.ny, C.pitch, F.pitch, C.cls, F.cls, Vol<T>(F), U<T>(F),
                                                        R<T>(F), Tmp<T>(F), R<T>(C), U<T>(C), S));
  else
    KL(dev::k_restrict_fused<T, false><<<grd, blk, 0, s>>>(C.nx, C.ny, C.pitch, F.pitch, C.cls, F.cls, Vol<T>(F), U<T>(F),
                                                         R<T>(F), Tmp<T>(F), R<T>(C), U<T>(C), S));
}

template <typename T>
void prolong_from(ccm_handle* H, DevLevel& F, DevLevel& C, cudaStream_t s) {
  if (F.ntiles == 0) return;
  dim3 blk(dev::TX, dev::TY);
  KL(launch_k(dev::k_prolong<T>, dim3(F.ntiles, H->nb), blk, 0, s, F.tiles, F.cls, F.nx, F.ny, F.pitch, C.pitch, U<T>(C),
              U<T>(F), F.npad, C.npad));
}

template <typename T>
void bottom(ccm_handle* H, DevLevel& B, cudaStream_t s) {
  if (B.nbc >= 256) {
    // column chunks over a cluster of CTAs (latency of the dense matrix-vector product)
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = dev::BOTTOM_SPLIT;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.gridDim = dim3(ceil_div(B.nbc, 32) * dev::BOTTOM_SPLIT, H->nb);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = t_pdl ? 2 : 1;
    KL(cudaLaunchKernelEx(&cfg, dev::k_bottom_split<T>, B.nbc, (const int32_t*)B.bot_cell, (const T*)Bot<T>(B),
                          (const T*)R<T>(B), U<T>(B), B.npad));
    return;
  }
  int nw = 8;
  size_t sm = std::max<size_t>(B.nbc, nw * 32) * sizeof(T);
  KL(launch_k(dev::k_bottom<T>, dim3(ceil_div(B.nbc, 32), H->nb), nw * 32, sm, s, B.nbc, B.bot_cell, Bot<T>(B), R<T>(B),
              U<T>(B), B.npad));
}

// the levels from m down to the bottom run as one launch of one thread-block cluster
template <typename T>
void coarse_cluster(ccm_handle* H, int m, cudaStream_t s) {
  const int M = (int)H->L.size() - 1;
  dev::CoarseParams<T> P{};
  P.nlev = M - m + 1;
  P.nu1 = H->par.nu1;
  P.nu2 = H->par.nu2;
  P.S = stencil<T>(H);
  for (int k = 0; k < P.nlev; ++k) {
    DevLevel& L = H->L[m + k];
    dev::CoarseLevel<T>& C = P.L[k];
    C.nx = L.nx; C.ny = L.ny; C.pitch = L.pitch; C.n2 = L.n2; C.nblk = L.nblk; C.nbc = L.nbc; C.W = L.W;
    C.cls = L.cls; C.vol = Vol<T>(L); C.r = R<T>(L);
    C.u[0] = sizeof(T) == 8 ? (T*)L.u64[0] : (T*)L.u32[0];
    C.u[1] = sizeof(T) == 8 ? (T*)L.u64[1] : (T*)L.u32[1];
    C.irr_cell = L.irr_cell; C.rowmap = L.rowmap; C.colf = L.ell_colf; C.par = L.ell_par; C.val = Ell<T>(L);
    C.blk = L.blk; C.blk_off = L.blk_off; C.inv = Inv<T>(L); C.bot_cell = L.bot_cell; C.bot = Bot<T>(L);
    P.cur[k] = sizeof(T) == 8 ? L.cur64 : L.cur32;
  }
  cudaLaunchConfig_t cfg{};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = H->coarse_ctas;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(H->coarse_ctas);
  cfg.blockDim = dim3(dev::COARSE_THREADS);
  cfg.dynamicSmemBytes = H->coarse_smem / 8 * sizeof(T);
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (H->cross) KL(cudaLaunchKernelEx(&cfg, dev::k_coarse_cluster<T, true>, P));
  else KL(cudaLaunchKernelEx(&cfg, dev::k_coarse_cluster<T, false>, P));
  const int flips = H->par.nu2 > 0 ? H->par.nu1 + H->par.nu2 : H->par.nu1;
  for (int k = 0; k + 1 < P.nlev; ++k)
    if (flips & 1) flip<T>(H->L[m + k]);
}

// cluster size for the coarse launch: 16 CTAs where the device schedules them, else 8
template <typename T, bool CROSS>
int coarse_cluster_ctas(size_t smem) {
  auto k = dev::k_coarse_cluster<T, CROSS>;
  if (smem > 48 * 1024 && cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  for (int cs : {16, 8}) {
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(dev::COARSE_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) == cudaSuccess && n >= 1) return cs;
  }
  cudaGetLastError();
  return 0;
}

// Alg. 2 from level m: solves L^(m) u = r^(m) approximately, u = U<T>(level m)
template <typename T>
void vcycle(ccm_handle* H, int m, cudaStream_t s, bool prolong_first = false) {
  const int M = (int)H->L.size() - 1;
  DevLevel& F = H->L[m];
  if (m == M) {
    bottom<T>(H, F, s);
    return;
  }
  DevLevel& C = H->L[m + 1];
  if (m >= H->coarse_first && M - m + 1 <= dev::MAXC) {
    if (prolong_first) prolong_from<T>(H, F, C, s);
    coarse_cluster<T>(H, m, s);
    return;
  }
  // prolong_first: the initial guess is u + P u^(m+1) (the FMG ascent); the first
  // pre-smoothing sweep reads it on the fly.  Otherwise a coarse level's iterate is 0 on entry
  // (the restriction cleared it), so its first persistent FP32 sweep does not read it; level
  // 0's first sweep gets the same request from the outer iteration
  if (prolong_first && H->par.nu1 == 0) prolong_from<T>(H, F, C, s);
  const bool persistent = F.smooth_ok[1] && H->persistent && H->par.smoother == 1 && H->par.ras_passes <= 1;
  for (int k = 0; k < H->par.nu1; ++k) {
    if (k == 0 && m > 0 && !prolong_first && sizeof(T) == 4 && persistent) H->zero_u_next = true;
    if (k > 0 || prolong_first) H->zero_u_next = false;
    if (k == 0 && prolong_first) smooth_step<T>(H, F, s, U<T>(C), C.pitch);
    else smooth_step<T>(H, F, s);
    H->zero_u_next = false;
  }
  restrict_to<T>(H, F, C, s);
  vcycle<T>(H, m + 1, s);
  if (H->par.nu2 == 0) {
    prolong_from<T>(H, F, C, s);
    return;
  }
  // the last inner cycle's last level-0 sweep may take the outer update u_hat += e
  const bool fold = m == 0 && H->fold_last;
  H->fold_next = fold && H->par.nu2 == 1;
  smooth_step<T>(H, F, s, U<T>(C), C.pitch);
  for (int k = 1; k < H->par.nu2; ++k) {
    H->fold_next = fold && k == H->par.nu2 - 1;
    smooth_step<T>(H, F, s);
  }
  H->fold_next = false;
}

// One FMG cycle (Sec. 4, the FMG figure) for L^(0) u = r^(0) from the zero guess: the
// right-hand side is restricted level by level to the bottom level (the restriction of
// r - L 0 with a zero iterate) and solved there; then every finer level runs one V-cycle
// (Alg. 2) from the prolonged coarse solution.  u = U<T>(level 0) on return.
template <typename T>
void fmg(ccm_handle* H, cudaStream_t s) {
  const int M = (int)H->L.size() - 1;
  DevLevel& L0 = H->L[0];
  cudaMemsetAsync(U<T>(L0), 0, (size_t)H->nb * L0.npad * sizeof(T), s);
  for (int m = 0; m < M; ++m) restrict_to<T>(H, H->L[m], H->L[m + 1], s);   // also zeroes u^(m+1)
  bottom<T>(H, H->L[M], s);
  for (int m = M - 1; m >= 0; --m) vcycle<T>(H, m, s, true);
}

// the regular cells' part of the outer residual runs in float-float arithmetic (about 48
// bits: good for relative residuals down to about 1e-11) when the tolerance allows, else in
// FP64
inline bool resid_float_float(const ccm_handle* H) { return H->par.rtol >= 1e-11; }

// mixed form: t = rhat - L uhat on level 0 into the FP32 right-hand side, max |t| into dnorm
void outer_residual32(ccm_handle* H, cudaStream_t s) {
  DevLevel& L = H->L[0];
  const int nb = H->nb;
  cudaMemsetAsync(H->dnorm, 0, nb * sizeof(unsigned long long), s);
  {
    ProfScope ps(H, CCM_PROF_RESID_FP64, s);
    const dim3 g(L.ntiles64, nb);
    if (resid_float_float(H)) {
      if (H->cross)
        KL(launch_k(dev::k_resid_ff<true>, g, 256, dev::Resid64Smem::bytes(true), s, H->tm_uhat, H->tm_rhat, L.tmcls,
                    L.tiles64, L.nx, L.pitch, L.r32, H->dnorm, H->ffs, H->derr, L.npad));
      else
        KL(launch_k(dev::k_resid_ff<false>, g, 256, dev::Resid64Smem::bytes(false), s, H->tm_uhat, H->tm_rhat, L.tmcls,
                    L.tiles64, L.nx, L.pitch, L.r32, H->dnorm, H->ffs, H->derr, L.npad));
    } else if (H->cross) {
      KL(launch_k(dev::k_resid64<true>, g, 256, dev::Resid64Smem::bytes(true), s, H->tm_uhat, H->tm_rhat,
                  L.tmcls, L.tiles64, L.nx, L.pitch, L.r32, H->dnorm, H->sep, H->derr, L.npad));
    } else {
      KL(launch_k(dev::k_resid64<false>, g, 256, dev::Resid64Smem::bytes(false), s, H->tm_uhat, H->tm_rhat,
                  L.tmcls, L.tiles64, L.nx, L.pitch, L.r32, H->dnorm, H->sep, H->derr, L.npad));
    }
  }
  if (L.n2)
    KL(launch_k(dev::k_rows_r32, dim3(ceil_div(L.n2, 128), nb), 128, 0, s, L.n2, L.W, L.irr_cell, L.ell_col, L.ell64,
                (const double*)H->uhat, (const double*)H->rhat, L.r32, H->dnorm, L.npad));
}

int check_level(ccm_handle* h, int level) {
  if (!h || level < 0 || level >= (int)h->L.size()) return CCM_EINVAL;
  return CCM_OK;
}

template <typename T>
void load_level(ccm_handle* h, DevLevel& L, const double* u, const double* r, cudaStream_t s) {
  dim3 pg(ceil_div(L.nx, 128), L.ny);
  cudaMemsetAsync(U<T>(L), 0, L.npad * sizeof(T), s);
  cudaMemsetAsync(Uother<T>(L), 0, L.npad * sizeof(T), s);
  cudaMemsetAsync(R<T>(L), 0, L.npad * sizeof(T), s);
  if (u) KL(dev::k_pack<T, double><<<pg, 128, 0, s>>>(L.nx, L.ny, L.pitch, L.cls, u, U<T>(L), 1.0));
  if (r) KL(dev::k_pack<T, double><<<pg, 128, 0, s>>>(L.nx, L.ny, L.pitch, L.cls, r, R<T>(L), L.h * L.h));
}

// tensor map over a padded level array (pitch x rows elements), zero fill outside; with
// depth > 0 it is 3-D over `depth` such arrays one after the other (the right-hand sides of
// a batch), box depth 1
bool make_tmap(CUtensorMap* map, void* base, int pitch, int rows, CUtensorMapDataType dt, size_t es, int bx, int by,
               int depth = 0) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return false;
    encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }
  const cuuint32_t rank = depth > 0 ? 3 : 2;
  cuuint64_t dims[3] = {(cuuint64_t)pitch, (cuuint64_t)rows, (cuuint64_t)std::max(depth, 1)};
  cuuint64_t strides[2] = {(cuuint64_t)pitch * es, (cuuint64_t)pitch * rows * es};
  cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = encode(map, dt, rank, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                      CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// the 68 x 36 halo tile box of the smoothing and restriction kernels, over `depth` arrays
bool make_tmap(CUtensorMap* map, void* base, int pitch, int rows, bool fp64, int depth) {
  return make_tmap(map, base, pitch, rows, fp64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                   fp64 ? 8 : 4, dev::HX, dev::HY, depth);
}

// device copies of level m's SMO-2 blocks (the ones of a previous call are given back)
int upload_blocks(ccm_handle* h, int m) {
  Arena& A = h->arena;
  const HostLevel& hl = h->H.levels[m];
  DevLevel& d = h->L[m];
  for (void* p : {(void*)d.order, (void*)d.blk, (void*)d.blk_off, (void*)d.inv64, (void*)d.inv32}) A.free(p);
  d.order = d.blk = nullptr;
  d.blk_off = nullptr;
  d.inv64 = nullptr;
  d.inv32 = nullptr;
  d.max_ext = d.max_core = 0;
  d.nblk = (int)hl.blk.size() / 4;
  if (!d.nblk) return CCM_OK;
  d.order = A.upload(hl.order);
  d.blk = A.upload(hl.blk);
  d.blk_off = A.upload(hl.blk_off);
  // 4 trailing zeros: bulk copies round a block's bytes up to a multiple of 16
  std::vector<double> g(hl.blk_inv.begin(), hl.blk_inv.end());
  g.resize(g.size() + 4, 0.0);
  d.inv64 = A.upload(g);
  std::vector<float> f(g.begin(), g.end());
  d.inv32 = A.upload(f);
  for (int b = 0; b < d.nblk; ++b) {
    d.max_ext = std::max(d.max_ext, hl.blk[4 * b + 3] - hl.blk[4 * b + 2]);
    d.max_core = std::max(d.max_core, hl.blk[4 * b + 1] - hl.blk[4 * b]);
  }
  if ((long)d.max_ext * (long)sizeof(double) > 48 * 1024) return CCM_EINVAL;
  return A.err == cudaSuccess ? CCM_OK : (A.err == cudaErrorMemoryAllocation ? CCM_ENOMEM : CCM_ECUDA);
}

// launch shape of a level's persistent sweep: two stages that hold a tile item or a block item,
// one CTA-wide item at a time (blocks with more core rows than one CTA covers keep the older
// path), as many CTAs as stay resident
void configure_sweep(ccm_handle* h, DevLevel& d, int nsm) {
  const size_t need = (size_t)d.max_ext * d.max_core * sizeof(double) + d.max_ext * sizeof(double) + 16;
  d.stage_blocks = d.nblk > 0 && need <= 200 * 1024;
  const int rows_per_cta = d.nblk >= 16 ? std::max(1, d.max_core) : 64;
  const bool one_chunk = d.nblk == 0 || d.max_core <= rows_per_cta;
  const int nitems = d.nblk + d.ntiles64;
  for (int k = 0; k < 2; ++k) d.smooth_ok[k] = false;
  for (int k = 0; k < 2 && d.tma && one_chunk && nitems > 0; ++k) {
    const size_t es = k == 0 ? sizeof(double) : sizeof(float);
    const size_t tile = k == 0 ? dev::TileStage<double>::bytes(true) : dev::TileStage<float>::bytes(true);
    const size_t blk = ((size_t)d.max_ext * d.max_core * es + 15) & ~(size_t)15;
    const size_t stage = (std::max(tile, blk) + 127) & ~(size_t)127;
    // two stages, then per extended row of a block: its residual, old value and cell
    const size_t smem = 2 * stage + 3 * (((size_t)std::max(1, d.max_ext) * es + 15) & ~(size_t)15);
    if (smem > 200 * 1024) continue;
    int occ = 0;
    if (k == 0) {
      auto fn = h->cross ? dev::k_smooth<double, true, true> : dev::k_smooth<double, false, true>;
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 256, smem);
      for (auto g : {h->cross ? dev::k_smooth<double, true, false> : dev::k_smooth<double, false, false>})
        cudaFuncSetAttribute(g, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    } else {
      auto fn = h->cross ? dev::k_smooth<float, true, true> : dev::k_smooth<float, false, true>;
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 256, smem);
      for (auto g : {h->cross ? dev::k_smooth<float, true, false> : dev::k_smooth<float, false, false>})
        cudaFuncSetAttribute(g, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    }
    if (occ < 1 || nsm < 1) continue;
    d.smooth_ok[k] = true;
    d.smooth_stage[k] = (uint32_t)stage;
    d.smooth_smem[k] = smem;
    d.smooth_grid[k] = std::min(nitems, nsm * occ);
    d.smooth_cap[k] = nsm * occ;
  }
  cudaGetLastError();
}

// Device copies of a host hierarchy (every level's arrays, work space, tensor maps, streams)
int upload_hierarchy(ccm_handle* h) {
  double w[5][5];
  regular_stencil(h->a, h->b, h->c, w);
  for (int k = 0; k < 25; ++k) {
    h->S64.w[k] = w[k / 5][k % 5];
    h->S32.w[k] = (float)w[k / 5][k % 5];
  }
  h->S64.omega_d = h->par.omega / w[2][2];
  h->S32.omega_d = (float)(h->par.omega / w[2][2]);
  {
    static const double lap[5] = {-1.0, 16.0, -30.0, 16.0, -1.0};
    static const double grad[5] = {1.0, -8.0, 0.0, 8.0, -1.0};
    for (int k = 0; k < 5; ++k) {
      h->S64.lx[k] = h->a * lap[k] / 12.0;
      h->S64.ly[k] = h->c * lap[k] / 12.0;
      h->S64.gx[k] = grad[k] / 12.0;
      h->S64.gy[k] = h->b * grad[k] / 12.0;
      h->S32.lx[k] = (float)h->S64.lx[k];
      h->S32.ly[k] = (float)h->S64.ly[k];
      h->S32.gx[k] = (float)h->S64.gx[k];
      h->S32.gy[k] = (float)h->S64.gy[k];
    }
    h->S64.cc = h->S64.lx[2] + h->S64.ly[2];
    h->S32.cc = (float)h->S64.cc;
  }

  Arena& A = h->arena;
  const int nl = (int)h->H.levels.size();
  h->L.resize(nl);
  for (int m = 0; m < nl; ++m) {
    HostLevel& hl = h->H.levels[m];
    DevLevel& d = h->L[m];
    d.nx = hl.nx;
    d.ny = hl.ny;
    d.pitch = hl.pitch;
    d.rows = hl.rows;
    d.npad = hl.npad();
    d.h = hl.h;
    d.ntiles = (int)hl.tiles.size() / 2;
    d.tiles = A.upload(hl.tiles);
    d.cls = A.upload(hl.cls);
    {
      std::vector<double> v64(hl.vol.begin(), hl.vol.end());
      d.vol64 = A.upload(v64);
      std::vector<float> v32(hl.vol.begin(), hl.vol.end());
      d.vol32 = A.upload(v32);
    }
    d.n2 = hl.n2;
    d.W = hl.W;
    if (hl.n2) {
      d.irr_cell = A.upload(hl.irr_cell);
      d.ell_col = A.upload(hl.ell_col);
      d.ell_colf = A.upload(hl.ell_colf);
      {
        std::vector<int32_t> rm(hl.npad(), -1);
        for (int r = 0; r < hl.n2; ++r) rm[hl.irr_cell[r]] = r;
        d.rowmap = A.upload(rm);
      }
      d.ell64 = A.upload(hl.ell_val);
      std::vector<float> f(hl.ell_val.begin(), hl.ell_val.end());
      d.ell32 = A.upload(f);
      d.nb = A.upload(hl.nb);
      d.seg = A.upload(hl.seg);
      d.res64 = A.alloc<double>(hl.n2);
      d.res32 = A.alloc<float>(hl.n2);
    }
    if (int rc = upload_blocks(h, m)) {
      A.release();
      return rc;
    }
    d.nbc = hl.nb_cells;
    if (d.nbc) {
      d.bot_cell = A.upload(hl.bot_cell);
      d.bot64 = A.upload(hl.bot_inv);
      std::vector<float> f(hl.bot_inv.begin(), hl.bot_inv.end());
      d.bot32 = A.upload(f);
    }
    if (!hl.tr_ptr.empty()) {
      d.ncolT = (int)hl.tr_cell.size();
      d.tr_ptr = A.upload(hl.tr_ptr);
      d.tr_cell = A.upload(hl.tr_cell);
      d.tr_row = A.upload(hl.tr_row);
      d.tr_val = A.upload(hl.tr_val);
    }
    d.ntiles64 = (int)hl.tiles64.size() / 2;
    if (d.ntiles64) d.tiles64 = A.upload(hl.tiles64);
    d.u64[0] = A.alloc<double>(d.npad);
    d.u64[1] = A.alloc<double>(d.npad);
    d.r64 = A.alloc<double>(d.npad);
    d.t64 = A.alloc<double>(d.npad);
    // the FP32 iterates and right-hand sides hold B right-hand sides one after the other
    d.u32[0] = A.alloc<float>(h->B * d.npad);
    d.u32[1] = A.alloc<float>(h->B * d.npad);
    d.r32 = A.alloc<float>(h->B * d.npad);
    d.t32 = A.alloc<float>(d.npad);
    // TMA-staged smoothing on the large levels (base addresses come from cudaMalloc, so
    // they are 256-byte aligned; the pitch is a multiple of 32 elements)
    d.tma = A.err == cudaSuccess && d.ntiles64 > 0 && d.nx >= 64;
    for (int b = 0; b < 2 && d.tma; ++b)
      d.tma = make_tmap(&d.tm64[b], d.u64[b], d.pitch, d.rows, true, 1) &&
              make_tmap(&d.tm32[b], d.u32[b], d.pitch, d.rows, false, h->B);
    d.tma = d.tma && make_tmap(&d.tmcls, d.cls, d.pitch, d.rows, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, dev::CLX, dev::HY) &&
            make_tmap(&d.tmv64, d.vol64, d.pitch, d.rows, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 8, dev::HX, dev::JY) &&
            make_tmap(&d.tmv32, d.vol32, d.pitch, d.rows, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, dev::HX, dev::JY) &&
            make_tmap(&d.tmr64, d.r64, d.pitch, d.rows, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 8, dev::HX, dev::JY, 1) &&
            make_tmap(&d.tmr32, d.r32, d.pitch, d.rows, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, dev::HX, dev::JY, h->B);
  }
  // SMO-2 blocks that fit in shared memory run as a bulk-staged kernel beside the sweep
  if (cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    A.release();
    return CCM_ECUDA;
  }
  cudaFuncSetAttribute(dev::k_blocks<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(dev::k_blocks<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device);
  for (int m = 0; m < nl; ++m) {
    DevLevel& d = h->L[m];
    configure_sweep(h, d, nsm);
    // parents of the fitted rows' regular columns (the prolongation read by SMO-2 residuals)
    if (m + 1 < nl && h->H.levels[m].n2) {
      const HostLevel& hf = h->H.levels[m];
      const int pc = h->L[m + 1].pitch;
      std::vector<int32_t> par(hf.ell_colf.size(), -1);
      for (size_t k = 0; k < par.size(); ++k) {
        const int f = hf.ell_colf[k];
        if (f >= 0) continue;
        const int q = f & 0x7fffffff, j = q / hf.pitch, i = q - j * hf.pitch;
        par[k] = ((j - 2) / 2 + 2) * pc + ((i - 2) / 2 + 2);
      }
      d.ell_par = A.upload(par);
    }
    // restriction tiles: fine 64 x 32 tiles with a non-empty fine cell or a non-empty coarse cell
    if (m + 1 < nl && d.tma) {
      const HostLevel& hf = h->H.levels[m];
      const HostLevel& hc = h->H.levels[m + 1];
      std::vector<int32_t> t;
      const int ax = (hf.nx + 63) / 64, ay = (hf.ny + 31) / 32;
      for (int b = 0; b < ay; ++b)
        for (int a = 0; a < ax; ++a) {
          bool any = false;
          for (int j = b * 32; j < std::min(hf.ny, b * 32 + 32) && !any; ++j)
            for (int i = a * 64; i < std::min(hf.nx, a * 64 + 64); ++i)
              if (hf.cls[hf.pad(i, j)] != 0 || hc.cls[hc.pad(i / 2, j / 2)] != 0) {
                any = true;
                break;
              }
          if (any) {
            t.push_back(a);
            t.push_back(b);
          }
        }
      d.ntiles64r = (int)t.size() / 2;
      if (d.ntiles64r) d.tiles64r = A.upload(t);
      // each restriction tile's irregular cells: (row, position in the tile)
      std::vector<int32_t> off(1, 0), rr;
      std::vector<int32_t> rowof(hf.npad(), -1);
      for (int r = 0; r < hf.n2; ++r) rowof[hf.irr_cell[r]] = r;
      for (int k = 0; k < d.ntiles64r; ++k) {
        const int a = t[2 * k], b = t[2 * k + 1];
        for (int j = b * 32; j < std::min(hf.ny, b * 32 + 32); ++j)
          for (int i = a * 64; i < std::min(hf.nx, a * 64 + 64); ++i) {
            const int r = rowof[hf.pad(i, j)];
            if (r < 0) continue;
            rr.push_back(r);
            rr.push_back((j - b * 32) * 64 + (i - a * 64));
          }
        off.push_back((int32_t)(rr.size() / 2));
      }
      if (d.ntiles64r) d.rr_off = A.upload(off);
      if (!rr.empty()) {
        d.rr = A.upload(rr);
        const int nr = (int)rr.size() / 2, W = hf.W;
        std::vector<int32_t> rq(2 * (size_t)nr), qc((size_t)W * nr);
        std::vector<double> qv((size_t)W * nr);
        for (int q = 0; q < nr; ++q) {
          const int r = rr[2 * q];
          rq[2 * q] = hf.irr_cell[r];
          rq[2 * q + 1] = rr[2 * q + 1];
          for (int k = 0; k < W; ++k) {
            qc[(size_t)k * nr + q] = hf.ell_col[(size_t)k * hf.n2 + r];
            qv[(size_t)k * nr + q] = hf.ell_val[(size_t)k * hf.n2 + r];
          }
        }
        std::vector<float> qv32(qv.begin(), qv.end());
        d.nrr = nr;
        d.rq = A.upload(rq);
        d.rq_col = A.upload(qc);
        d.rq_val64 = A.upload(qv);
        d.rq_val32 = A.upload(qv32);
      }
      // the first post-smoothing sweep reads u + P uc through two more boxes
      DevLevel& c = h->L[m + 1];
      d.tma_pro = true;
      for (int b = 0; b < 2 && d.tma_pro; ++b)
        d.tma_pro = make_tmap(&d.tmuc64[b], c.u64[b], c.pitch, c.rows, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 8, dev::UCX, dev::UCY, 1) &&
                    make_tmap(&d.tmuc32[b], c.u32[b], c.pitch, c.rows, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, dev::UCX, dev::UCY,
                              h->B);
      // the persistent restriction: two stages of u, r, class bytes and volumes per tile
      for (int k = 0; k < 2 && d.ntiles64r > 0; ++k) {
        const uint32_t stage = k == 0 ? dev::RestrictStage<double>::bytes : dev::RestrictStage<float>::bytes;
        const size_t smem = 2 * (size_t)stage;
        int occ = 0;
        if (k == 0) {
          auto fn = h->cross ? dev::k_restrict_p<double, true> : dev::k_restrict_p<double, false>;
          cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 256, smem);
        } else {
          auto fn = h->cross ? dev::k_restrict_p<float, true> : dev::k_restrict_p<float, false>;
          cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 256, smem);
        }
        if (occ < 1 || nsm < 1) continue;
        d.restrict_ok[k] = true;
        d.restrict_stage[k] = stage;
        d.restrict_grid[k] = std::min(d.ntiles64r, nsm * occ);
        d.restrict_cap[k] = nsm * occ;
      }
      cudaGetLastError();
    }
  }
  // the cluster launch takes over from the first level with at most coarse_n cells a side
  // (block-Jacobi smoother only: its sweeps read nothing but the old iterate)
  if (h->par.coarse_n > 0 && h->par.smoother == 1 && h->par.ras_passes <= 1) {
    int first = -1;
    for (int m = 1; m < nl; ++m)
      if (h->L[m].nx <= h->par.coarse_n && h->L[m].ny <= h->par.coarse_n) {
        first = m;
        break;
      }
    if (first > 0 && nl - first <= dev::MAXC) {
      int ext = std::max(1, h->L[nl - 1].nbc);
      for (int m = first; m < nl; ++m) ext = std::max(ext, h->L[m].max_ext);
      h->coarse_smem = (size_t)ext * sizeof(double);
      const int c64 = h->cross ? coarse_cluster_ctas<double, true>(h->coarse_smem)
                               : coarse_cluster_ctas<double, false>(h->coarse_smem);
      const int c32 = h->cross ? coarse_cluster_ctas<float, true>(h->coarse_smem / 2)
                               : coarse_cluster_ctas<float, false>(h->coarse_smem / 2);
      h->coarse_ctas = std::min(c64, c32);
      if (h->coarse_ctas > 0) h->coarse_first = first;
    }
  }
  h->rhat = A.alloc<double>(h->B * h->L[0].npad);
  h->uhat = A.alloc<double>(h->B * h->L[0].npad);
  {
    static const double lap[5] = {-1.0, 16.0, -30.0, 16.0, -1.0};
    static const double grad[5] = {1.0, -8.0, 0.0, 8.0, -1.0};
    for (int k = 0; k < 5; ++k) {
      h->sep.lx[k] = h->a * lap[k] / 12.0;
      h->sep.ly[k] = h->c * lap[k] / 12.0;
      h->sep.gx[k] = grad[k] / 12.0;
      h->sep.gy[k] = h->b * grad[k] / 12.0;
    }
    h->sep.cc = h->sep.lx[2] + h->sep.ly[2];
    auto split = [](double v, float& hi, float& lo) {
      hi = (float)v;
      lo = (float)(v - (double)hi);
    };
    split(h->a / 12.0, h->ffs.ah, h->ffs.al);
    split(h->c / 12.0, h->ffs.ch, h->ffs.cl);
    split(h->b / 144.0, h->ffs.bh, h->ffs.bl);
    const DevLevel& d0 = h->L[0];
    cudaFuncSetAttribute(dev::k_resid64<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, dev::Resid64Smem::bytes(true));
    cudaFuncSetAttribute(dev::k_resid64<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, dev::Resid64Smem::bytes(false));
    cudaFuncSetAttribute(dev::k_resid_ff<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, dev::Resid64Smem::bytes(true));
    cudaFuncSetAttribute(dev::k_resid_ff<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, dev::Resid64Smem::bytes(false));
    h->fused_outer = A.err == cudaSuccess && d0.tma && d0.ntiles64 > 0 &&
                     make_tmap(&h->tm_uhat, h->uhat, d0.pitch, d0.rows, true, h->B) &&
                     make_tmap(&h->tm_rhat, h->rhat, d0.pitch, d0.rows, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 8, dev::HX, dev::JY,
                               h->B);
  }
  if (h->par.precision == CCM_MIXED && h->par.krylov > 0 && h->fused_outer) {
    h->kry_m = h->par.krylov;
    for (int i = 0; i <= h->kry_m; ++i) h->kv[i] = A.alloc<float>(h->L[0].npad);
    for (int i = 0; i < h->kry_m; ++i) h->kz[i] = A.alloc<float>(h->L[0].npad);
    h->ks = A.alloc<dev::KryScalars>(1);
  }
  h->dnorm = A.alloc<unsigned long long>(2 * h->B);   // [0, B) residual norms, [B, 2B) ||r_hat||
  h->derr = A.alloc<int>(1);
  if (A.err != cudaSuccess) {
    A.release();
    return A.err == cudaErrorMemoryAllocation ? CCM_ENOMEM : CCM_ECUDA;
  }
  if (cudaMallocHost(&h->hnorm, 2 * h->B * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMallocHost(&h->herr, sizeof(int)) != cudaSuccess) {
    A.release();
    return CCM_ECUDA;
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    A.release();
    return CCM_ECUDA;
  }
  return CCM_OK;
}

}  // namespace

// ================================================================ C ABI

extern "C" {

int ccm_default_params(ccm_params* p) {
  if (!p) return CCM_EINVAL;
  p->omega = 0.7;
  p->nu1 = 3;
  p->nu2 = 3;
  p->theta = 0.3;
  p->coarsest = 16;
  p->precision = CCM_MIXED;
  p->rtol = 1e-10;
  p->max_iter = 100;
  p->ras_passes = 1;
  p->ras_block = 64;
  p->ras_overlap = 24;
  p->nthreads = 0;
  p->ras_exact = 0;
  p->inner_cycles = 3;
  p->smoother = 1;
  p->coarse_n = 0;
  p->batch = 1;
  p->cycle = 0;
  p->setup_device = 1;
  p->krylov = 0;
  return CCM_OK;
}

const char* ccm_strerror(int code) {
  switch (code) {
    case CCM_OK: return "ok";
    case CCM_EINVAL: return "invalid argument";
    case CCM_EGEOM: return "invalid or degenerate geometry";
    case CCM_EPLG: return "no poised PLG stencil within the search radius";
    case CCM_ESINGULAR: return "singular block or bottom factorisation";
    case CCM_ENOCONV: return "not converged within max_iter";
    case CCM_ETIMEOUT: return "bounded device wait ran out";
    case CCM_ECUDA: return "CUDA runtime error";
    case CCM_ENOMEM: return "out of memory";
    case CCM_ENOTFINITE: return "residual is not finite";
    case CCM_ETOOLARGE: return "grid exceeds the fixed scratch of the allocation-free entry point";
    default: return "unknown error";
  }
}

int ccm_setup(const ccm_problem* prob, const ccm_params* params, ccm_handle** out) {
  if (!prob || !out) return CCM_EINVAL;
  *out = nullptr;
  if (int rc = check_problem(*prob)) return rc;
  ccm_params par;
  ccm_default_params(&par);
  if (params) par = *params;
  if (par.nu1 < 0 || par.nu2 < 0 || par.coarsest < 4 || par.ras_passes < 0 || par.ras_block < 8 ||
      par.ras_block > 128 || par.ras_overlap < 0 || par.ras_overlap > 64 || par.max_iter < 0 ||
      par.ras_exact < 0 || par.ras_exact > 6000 || par.inner_cycles < 1 || par.inner_cycles > 16 || par.smoother < 0 || par.smoother > 1 || par.coarse_n < 0 ||
      par.batch < 1 || par.batch > 4096 || par.cycle < 0 || par.cycle > 1 || par.krylov < 0 ||
      par.krylov > dev::KRY_MAXM ||
      !(par.theta >= 0 && par.theta < 1) || (par.precision != CCM_FP64 && par.precision != CCM_MIXED))
    return CCM_EINVAL;
  auto t0 = std::chrono::steady_clock::now();
  std::unique_ptr<ccm_handle> h(new ccm_handle());
  h->par = par;
  h->B = par.precision == CCM_MIXED ? par.batch : 1;
  h->a = prob->a;
  h->b = prob->b;
  h->c = prob->c;
  h->cross = prob->b != 0.0;
  cudaGetDevice(&h->device);
  std::string err;
  int rc;
  try {
    std::unique_ptr<FitBatcher> fb;
    std::unique_ptr<CentreClassifier> cc;
    if (par.setup_device) {
      fb = make_device_fitter();
      cc = make_device_classifier();
    }
    rc = build_hierarchy(*prob, par, h->H, err, fb.get(), cc.get());
  } catch (const std::bad_alloc&) {
    return CCM_ENOMEM;
  }
  if (rc) return rc;
  auto t_up = std::chrono::steady_clock::now();
  rc = upload_hierarchy(h.get());
  if (rc) return rc;
  h->info.setup_upload_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_up).count();
  h->info.setup_geometry_ms = h->H.ms_geometry;
  h->info.setup_fits_ms = h->H.ms_fits;
  h->info.setup_blocks_ms = h->H.ms_blocks;
  h->info.setup_bottom_ms = h->H.ms_bottom;
  const int nl = (int)h->H.levels.size();
  Arena& A = h->arena;
  // info
  ccm_info& I = h->info;
  const CutLevel& c0 = h->H.cut[0];
  I.nx = prob->nx;
  I.ny = prob->ny;
  I.levels = nl;
  I.n_cells = 0;
  I.n_regular = 0;
  for (long q = 0; q < (long)prob->nx * prob->ny; ++q)
    if (c0.status[q] != ST_EMPTY) ++I.n_cells;
  I.n_irregular = h->H.levels[0].n2;
  I.n_regular = I.n_cells - I.n_irregular;
  I.n_segments = h->H.nseg;
  I.device_bytes = A.bytes;
  I.plg_cond_max = h->H.cond_max;
  // batching needs every launch of an outer iteration to take its right-hand side from the
  // grid: the persistent sweep and restriction on every TMA level, the fused outer residual,
  // the block-Jacobi smoother and no cluster cycle
  {
    bool ok = h->B > 1 && h->fused_outer && h->persistent && par.smoother == 1 && par.ras_passes <= 1 &&
              h->coarse_first >= nl && h->kry_m == 0;
    for (int m = 0; m < nl && ok; ++m) {
      const DevLevel& d = h->L[m];
      if (!d.tma) continue;
      if (d.nblk + d.ntiles64 > 0 && !d.smooth_ok[1]) ok = false;
      if (m + 1 < nl && d.ntiles64r > 0 && !d.restrict_ok[1]) ok = false;
    }
    h->bmax = ok ? h->B : 1;
    I.batch = h->bmax;
  }
  I.setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  *out = h.release();
  return CCM_OK;
}

int ccm_query(const ccm_handle* h, ccm_info* info) {
  if (!h || !info) return CCM_EINVAL;
  *info = h->info;
  return CCM_OK;
}

int ccm_cell_map(const ccm_handle* h, int8_t* status, int32_t* owner, int8_t* regular, double* vol) {
  if (!h) return CCM_EINVAL;
  const CutLevel& c = h->H.cut[0];
  const HostLevel& L = h->H.levels[0];
  long n = (long)c.nx * c.ny;
  if (status) std::memcpy(status, c.status.data(), n);
  if (owner) std::memcpy(owner, c.owner.data(), n * sizeof(int32_t));
  if (vol) std::memcpy(vol, c.vol.data(), n * sizeof(double));
  if (regular)
    for (int j = 0; j < c.ny; ++j)
      for (int i = 0; i < c.nx; ++i) regular[(long)j * c.nx + i] = L.cls[L.pad(i, j)] == 1 ? 1 : 0;
  return CCM_OK;
}

int ccm_boundary_segments(const ccm_handle* h, int32_t* cell, int32_t* bc, double* length) {
  if (!h) return CCM_EINVAL;
  const CutLevel& c = h->H.cut[0];
  for (size_t s = 0; s < c.segs.size(); ++s) {
    if (cell) cell[s] = c.segs[s];
    if (bc) bc[s] = c.seg_bc[s];
    if (length) length[s] = c.bm0[s][0] * c.h;
  }
  return CCM_OK;
}

int ccm_level_rows(const ccm_handle* h, int level, int64_t* n_rows, int32_t* cell, int32_t* cols, double* beta,
                   double* nb, int32_t* seg) {
  if (!h || level < 0 || level >= (int)h->H.levels.size()) return CCM_EINVAL;
  if (n_rows) *n_rows = h->H.levels[level].n2;
  return hierarchy_rows(h->H, level, cell, cols, beta, nb, seg);
}

int ccm_boundary_robin(const ccm_handle* h, double* gamma) {
  if (!h || !gamma) return CCM_EINVAL;
  const CutLevel& c = h->H.cut[0];
  for (size_t s = 0; s < c.segs.size(); ++s) {
    gamma[2 * s] = c.seg_gamma[s][0];
    gamma[2 * s + 1] = c.seg_gamma[s][1];
  }
  return CCM_OK;
}

int ccm_quadrature(const ccm_handle* h, int64_t* n_cell_nodes, int64_t* n_bdry_nodes, int32_t* cell_of,
                   double* cxy, double* cw, int32_t* seg_of, double* bxy, double* bw, double* bn) {
  if (!h || !n_cell_nodes || !n_bdry_nodes) return CCM_EINVAL;
  std::vector<int32_t> cc, ss;
  std::vector<double> xy, w, bxy_, bw_, bn_;
  cell_quadrature(h->H.cut[0], cc, xy, w);
  boundary_quadrature(h->H.cut[0], ss, bxy_, bw_, bn_);
  if (cell_of && cxy && cw) {
    if (*n_cell_nodes < (int64_t)cc.size()) return CCM_EINVAL;
    std::memcpy(cell_of, cc.data(), cc.size() * sizeof(int32_t));
    std::memcpy(cxy, xy.data(), xy.size() * sizeof(double));
    std::memcpy(cw, w.data(), w.size() * sizeof(double));
  }
  if (seg_of && bxy && bw && bn) {
    if (*n_bdry_nodes < (int64_t)ss.size()) return CCM_EINVAL;
    std::memcpy(seg_of, ss.data(), ss.size() * sizeof(int32_t));
    std::memcpy(bxy, bxy_.data(), bxy_.size() * sizeof(double));
    std::memcpy(bw, bw_.data(), bw_.size() * sizeof(double));
    std::memcpy(bn, bn_.data(), bn_.size() * sizeof(double));
  }
  *n_cell_nodes = (int64_t)cc.size();
  *n_bdry_nodes = (int64_t)ss.size();
  return CCM_OK;
}

int ccm_cell_averages(const ccm_handle* h, ccm_field_fn f, void* ctx, double* out) {
  if (!h || !f || !out) return CCM_EINVAL;
  cell_averages(h->H.cut[0], f, ctx, out);
  return CCM_OK;
}

int ccm_boundary_averages(const ccm_handle* h, ccm_grad_fn g, void* ctx, double* out) {
  if (!h || !g || !out) return CCM_EINVAL;
  boundary_averages(h->H.cut[0], g, ctx, out);
  return CCM_OK;
}

int ccm_apply(ccm_handle* h, const double* u, const double* g, double* out, int nrhs, void* stream) {
  if (!h || !u || !out || nrhs < 1) return CCM_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  DevLevel& L = h->L[0];
  const long nu = (long)L.nx * L.ny;
  dim3 pg(ceil_div(L.nx, 128), L.ny);
  for (int k = 0; k < nrhs; ++k) {
    KL(dev::k_pack<double, double><<<pg, 128, 0, s>>>(L.nx, L.ny, L.pitch, L.cls, u + k * nu, L.t64, 1.0));
    launch_regular<double>(h, L, L.t64, nullptr, L.u64[1 - L.cur64], false, s);
    if (L.n2)
      KL(launch_k(dev::k_rows<double, double, false, true>, ceil_div(L.n2, 128), 128, 0, s, 
          L.n2, L.W, L.irr_cell, L.ell_col, L.ell64, L.t64, nullptr, L.u64[1 - L.cur64], L.nb, L.seg,
          g ? g + (long)k * h->info.n_segments : nullptr));
    KL(dev::k_unpack<double><<<pg, 128, 0, s>>>(L.nx, L.ny, L.pitch, L.cls, L.u64[1 - L.cur64], out + k * nu,
                                             1.0 / (L.h * L.h)));
  }
  CCM_CUDA(cudaGetLastError());
  return CCM_OK;
}

}  // extern "C"

// Scratch of ccm_apply_noalloc: two padded FP64 grids, held by every device that loads the
// library.  Host code only ever uses the device address looked up below.
static __device__ __align__(256) double g_noalloc_scratch[2 * CCM_NOALLOC_MAX_PADDED];

namespace {
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[256] = {nullptr};

// device address of the scratch array on the current device (looked up once per device)
int noalloc_scratch(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return CCM_ECUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return CCM_ECUDA;
    g_noalloc_ptr[dev] = (double*)p;
  }
  *out = g_noalloc_ptr[dev];
  return CCM_OK;
}
}  // namespace

extern "C" {

int ccm_apply_noalloc(const ccm_handle* hc, const double* u, const double* g, double* out, void* stream) {
  if (!hc || !u || !out) return CCM_EINVAL;
  ccm_handle* h = const_cast<ccm_handle*>(hc);
  const DevLevel& L = h->L[0];
  if (L.npad > CCM_NOALLOC_MAX_PADDED) return CCM_ETOOLARGE;
  // the scratch address below is the current device's; the handle's arrays live on h->device
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return CCM_ECUDA;
  if (cur != h->device) return CCM_EINVAL;
  double* scratch = nullptr;
  int rc = noalloc_scratch(&scratch);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  double* up = scratch;                              // padded u
  double* op = scratch + CCM_NOALLOC_MAX_PADDED;     // padded L u + N g
  CCM_CUDA(cudaMemsetAsync(up, 0, L.npad * sizeof(double), s));
  CCM_CUDA(cudaMemsetAsync(op, 0, L.npad * sizeof(double), s));
  dim3 pg(ceil_div(L.nx, 128), L.ny);
  KL(dev::k_pack<double, double><<<pg, 128, 0, s>>>(L.nx, L.ny, L.pitch, L.cls, u, up, 1.0));
  if (L.ntiles) {
    dim3 blk(dev::TX, dev::TY);
    if (h->cross)
      KL(launch_k(dev::k_regular<double, true, false>, L.ntiles, blk, 0, s, L.tiles, L.cls, L.nx, L.ny, L.pitch, up, nullptr, op, h->S64));
    else
      KL(launch_k(dev::k_regular<double, false, false>, L.ntiles, blk, 0, s, L.tiles, L.cls, L.nx, L.ny, L.pitch, up, nullptr, op, h->S64));
  }
  if (L.n2)
    KL(launch_k(dev::k_rows<double, double, false, true>, ceil_div(L.n2, 128), 128, 0, s, 
        L.n2, L.W, L.irr_cell, L.ell_col, L.ell64, up, nullptr, op, L.nb, L.seg, g));
  KL(dev::k_unpack<double><<<pg, 128, 0, s>>>(L.nx, L.ny, L.pitch, L.cls, op, out, 1.0 / (L.h * L.h)));
  CCM_CUDA(cudaGetLastError());
  return CCM_OK;
}

int ccm_apply_T(ccm_handle* h, const double* v, double* out_u, double* out_g, int nrhs, void* stream) {
  if (!h || !v || nrhs < 1 || (!out_u && !out_g)) return CCM_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  DevLevel& L = h->L[0];
  const long nu = (long)L.nx * L.ny;
  dim3 pg(ceil_div(L.nx, 128), L.ny);
  const double sc = 1.0 / (L.h * L.h);
  for (int k = 0; k < nrhs; ++k) {
    KL(dev::k_pack<double, double><<<pg, 128, 0, s>>>(L.nx, L.ny, L.pitch, L.cls, v + k * nu, L.t64, 1.0));
    if (out_u) {
      double* o = L.u64[1 - L.cur64];
      dim3 blk(dev::TX, dev::TY);
      if (L.ntiles) {
        if (h->cross) KL(dev::k_regular_T<true><<<L.ntiles, blk, 0, s>>>(L.tiles, L.cls, L.nx, L.ny, L.pitch, L.t64, o, h->S64));
        else KL(dev::k_regular_T<false><<<L.ntiles, blk, 0, s>>>(L.tiles, L.cls, L.nx, L.ny, L.pitch, L.t64, o, h->S64));
      }
      if (L.ncolT)
        KL(dev::k_rows_T<<<ceil_div(L.ncolT, 128), 128, 0, s>>>(L.ncolT, L.tr_ptr, L.tr_cell, L.tr_row, L.tr_val,
                                                            L.irr_cell, L.t64, o));
      KL(dev::k_unpack<double><<<pg, 128, 0, s>>>(L.nx, L.ny, L.pitch, L.cls, o, out_u + k * nu, sc));
    }
    if (out_g && L.n2)
      KL(dev::k_bnd_T<<<ceil_div(L.n2, 128), 128, 0, s>>>(L.n2, L.irr_cell, L.nb, L.seg, L.t64,
                                                      out_g + (long)k * h->info.n_segments, sc));
  }
  CCM_CUDA(cudaGetLastError());
  return CCM_OK;
}

// The correction of one mixed outer iteration by GMRES(m) on L e = r32 with the inner FP32
// V-cycles as right preconditioner (see krylov.cuh); u_hat += e.  Level-0 FP32 vectors only,
// scalars in device memory, no host synchronisation.
static void krylov_correction(ccm_handle* h, cudaStream_t s) {
  DevLevel& L = h->L[0];
  const int m = h->kry_m, nt = L.ntiles;
  dev::KryScalars* S = h->ks;
  dev::KryVecs V{}, Z{}, R{};
  for (int i = 0; i <= m; ++i) V.v[i] = h->kv[i];
  for (int i = 0; i < m; ++i) Z.v[i] = h->kz[i];
  R.v[0] = L.r32;
  const int KT = dev::KRY_THREADS, KG = dev::KRY_GRID;
  const int32_t* tl = L.tiles;
  const uint8_t* cl = L.cls;
  cudaMemsetAsync(reinterpret_cast<char*>(S) + offsetof(dev::KryScalars, H), 0, sizeof(S->H), s);
  // beta = ||r||_2, v_0 = r / beta, which is also the first preconditioner input
  KL(launch_k(dev::k_kdot, KG, KT, 0, s, tl, nt, L.nx, L.ny, L.pitch, (const float*)L.r32, R, 1, S));
  KL(launch_k(dev::k_kreduce, 1, KT, 0, s, 1, 2, 0, m, S));
  KL(launch_k(dev::k_kscale, KG, KT, 0, s, tl, nt, L.nx, L.ny, L.pitch, cl, (const float*)L.r32, h->kv[0], L.r32,
              (const dev::KryScalars*)S));
  for (int j = 0; j < m; ++j) {
    // z_j = M v_j: the inner cycles from a zero guess on the right-hand side r32 = v_j
    cudaMemsetAsync(L.u32[L.cur32], 0, L.npad * sizeof(float), s);
    for (int c = 0; c < std::max(1, h->par.inner_cycles); ++c) {
      ProfScope ps(h, CCM_PROF_VCYCLE, s);
      if (c == 0 && h->par.cycle == 1) fmg<float>(h, s);
      else vcycle<float>(h, 0, s);
    }
    const float* z = L.u32[L.cur32];
    float* w = h->kv[j + 1];
    // w = L z (regular stencil, then the fitted rows), z kept as z_j
    if (h->cross)
      KL(launch_k(dev::k_kapply<true>, nt, KT, 0, s, tl, L.nx, L.ny, L.pitch, cl, z, w, h->kz[j], h->S32));
    else
      KL(launch_k(dev::k_kapply<false>, nt, KT, 0, s, tl, L.nx, L.ny, L.pitch, cl, z, w, h->kz[j], h->S32));
    if (L.n2)
      KL(launch_k(dev::k_rows<float, float, false, true>, ceil_div(L.n2, 128), 128, 0, s, L.n2, L.W,
                  (const int32_t*)L.irr_cell, (const int32_t*)L.ell_col, (const float*)L.ell32, z, (const float*)nullptr, w,
                  (const double*)nullptr, (const int32_t*)nullptr, (const double*)nullptr));
    // classical Gram-Schmidt against v_0 .. v_j twice, each subtraction fused with the next
    // reduction: the second pass's dot products, then ||w||^2
    KL(launch_k(dev::k_kdot, KG, KT, 0, s, tl, nt, L.nx, L.ny, L.pitch, (const float*)w, V, j + 1, S));
    KL(launch_k(dev::k_kreduce, 1, KT, 0, s, j + 1, 0, j, m, S));
    KL(launch_k(dev::k_ksubdot, KG, KT, 0, s, tl, nt, L.nx, L.ny, L.pitch, cl, w, V, j + 1, false, S));
    KL(launch_k(dev::k_kreduce, 1, KT, 0, s, j + 1, 0, j, m, S));
    KL(launch_k(dev::k_ksubdot, KG, KT, 0, s, tl, nt, L.nx, L.ny, L.pitch, cl, w, V, j + 1, true, S));
    // h_{j+1,j} = ||w||, v_{j+1} = w / h_{j+1,j} (and the next preconditioner input)
    KL(launch_k(dev::k_kreduce, 1, KT, 0, s, 1, 1, j, m, S));
    KL(launch_k(dev::k_kscale, KG, KT, 0, s, tl, nt, L.nx, L.ny, L.pitch, cl, (const float*)w, w,
                j + 1 < m ? L.r32 : (float*)nullptr, (const dev::KryScalars*)S));
  }
  KL(launch_k(dev::k_klsq, 1, 32, 0, s, m, S));
  KL(launch_k(dev::k_kupdate, KG, KT, 0, s, tl, nt, L.nx, L.ny, L.pitch, cl, Z, m, (const dev::KryScalars*)S, h->uhat));
}

// One outer iteration on the stream (also the body captured into the iteration graph):
// mixed: FP32 V-cycles on the FP32 image of the FP64 residual, u_hat += e, new FP64 residual;
// fp64:  one FP64 V-cycle in place, new FP64 residual; then the residual norm to the host.
// one outer iteration on stream s; with to_host the residual norm and the error word are
// copied to the handle's pinned host words at its end
static void iteration_body(ccm_handle* h, bool fp64, cudaStream_t s, bool to_host = true) {
  DevLevel& L = h->L[0];
  const long np = L.npad;
  double* ucur;
  if (fp64) {
    double* start = L.u64[L.cur64];
    {
      ProfScope ps(h, CCM_PROF_VCYCLE, s);
      vcycle<double>(h, 0, s);
    }
    if (L.u64[L.cur64] != start) {
      cudaMemcpyAsync(start, L.u64[L.cur64], np * sizeof(double), cudaMemcpyDeviceToDevice, s);
      L.cur64 = 1 - L.cur64;
    }
    ucur = start;
  } else if (h->fused_outer && h->kry_m > 0) {
    // r32 holds the FP32 image of the residual; e by GMRES(m) preconditioned by the cycles
    krylov_correction(h, s);
    outer_residual32(h, s);
    if (!to_host) return;
    cudaMemcpyAsync(h->hnorm, h->dnorm, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(h->herr, h->derr, sizeof(int), cudaMemcpyDeviceToHost, s);
    return;
  } else if (h->fused_outer) {
    // r32 holds the FP32 image of the residual (previous iteration or the initial one).  Where
    // level 0 runs the persistent sweep, its first sweep starts from the zero correction
    // without reading it (no clearing pass), and the last one adds its new values to u_hat
    // (no separate update pass)
    const bool persistent0 = L.smooth_ok[1] && h->persistent && h->par.smoother == 1 && h->par.ras_passes <= 1;
    const bool zero_first = persistent0 && h->par.nu1 >= 1 && h->par.cycle == 0;
    if (!zero_first) cudaMemsetAsync(L.u32[L.cur32], 0, h->nb * np * sizeof(float), s);
    const int ncyc = std::max(1, h->par.inner_cycles);
    h->folded = false;
    for (int c = 0; c < ncyc; ++c) {
      ProfScope ps(h, CCM_PROF_VCYCLE, s);
      h->zero_u_next = c == 0 && zero_first;
      h->fold_last = c == ncyc - 1 && persistent0;
      if (c == 0 && h->par.cycle == 1) fmg<float>(h, s);     // FMG, then V-cycles from its result
      else vcycle<float>(h, 0, s);
      h->zero_u_next = h->fold_last = false;
    }
    if (!h->folded) {
      dim3 blk(dev::TX, dev::TY);
      KL(launch_k(dev::k_axpy_tiles, dim3(L.ntiles, h->nb), blk, 0, s, L.tiles, L.cls, L.nx, L.ny, L.pitch,
                  (const float*)L.u32[L.cur32], h->uhat, L.npad));
    }
    h->folded = false;
    outer_residual32(h, s);
    if (!to_host) return;
    cudaMemcpyAsync(h->hnorm, h->dnorm, h->nb * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(h->herr, h->derr, sizeof(int), cudaMemcpyDeviceToHost, s);
    return;
  } else {
    KL(launch_k(dev::k_to_float, std::min(ceil_div(np, 256), 4096), 256, 0, s, np, L.t64, L.r32));
    cudaMemsetAsync(L.u32[L.cur32], 0, np * sizeof(float), s);
    for (int c = 0; c < std::max(1, h->par.inner_cycles); ++c) {
      ProfScope ps(h, CCM_PROF_VCYCLE, s);
      if (c == 0 && h->par.cycle == 1) fmg<float>(h, s);     // FMG, then V-cycles from its result
      else vcycle<float>(h, 0, s);
    }
    KL(launch_k(dev::k_axpy<float>, std::min(ceil_div(np, 256), 4096), 256, 0, s, np, L.cls, L.u32[L.cur32], h->uhat));
    ucur = h->uhat;
  }
  {
    ProfScope ps(h, CCM_PROF_RESID_FP64, s);
    launch_regular<double>(h, L, ucur, h->rhat, L.t64, true, s);
  }
  if (L.n2)
    KL(launch_k(dev::k_rows<double, double, true, true>, ceil_div(L.n2, 128), 128, 0, s, 
        L.n2, L.W, L.irr_cell, L.ell_col, L.ell64, ucur, h->rhat, L.t64, nullptr, nullptr, nullptr));
  cudaMemsetAsync(h->dnorm, 0, sizeof(unsigned long long), s);
  KL(launch_k(dev::k_absmax<double>, std::min(ceil_div(np, 256), 1216), 256, 0, s, np, L.cls, L.t64, h->dnorm, 0L));
  if (!to_host) return;
  cudaMemcpyAsync(h->hnorm, h->dnorm, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(h->herr, h->derr, sizeof(int), cudaMemcpyDeviceToHost, s);
}

static int capture_iteration(ccm_handle* h, bool fp64, cudaStream_t user) {
  ccm_handle::Graph& G = h->graph[fp64 ? 1 : 0];
  if (G.exec && G.nb == h->nb) return CCM_OK;
  if (G.exec) {        // captured for another batch size
    CCM_CUDA(cudaStreamSynchronize(user));
    cudaGraphExecDestroy(G.exec);
    G.exec = nullptr;
    G.prof_pairs.clear();
  }
  if (!h->cap_stream) CCM_CUDA(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  CCM_CUDA(cudaStreamSynchronize(user));
  cudaStream_t s = h->cap_stream;
  // the body leaves every ping-pong buffer where it found it only for an even number of
  // sweeps per level; odd counts are handled inside the body (fp64) or by resetting the
  // level-0 FP32 buffer at the start of every replay (mixed)
  const int cur64 = h->L[0].cur64;
  cudaGraph_t graph;
  CCM_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  h->capturing = true;
  size_t ev0 = h->gprof_ev.size();
  long long l0 = g_launches.load();
  iteration_body(h, fp64, s);
  G.launches = g_launches.load() - l0;
  g_launches.fetch_sub(G.launches);
  h->capturing = false;
  cudaError_t e = cudaStreamEndCapture(s, &graph);
  if (e != cudaSuccess) return CCM_ECUDA;
  for (size_t k = ev0; k < h->gprof_ev.size(); k += 2) G.prof_pairs.push_back((int)k);
  e = cudaGraphInstantiate(&G.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    G.exec = nullptr;
    return CCM_ECUDA;
  }
  h->L[0].cur64 = cur64;
  G.u0 = fp64 ? h->L[0].u64[cur64] : h->uhat;
  G.nb = h->nb;
  return CCM_OK;
}

static void drop_graphs(ccm_handle* h) {
  for (auto& G : h->graph) {
    if (G.exec) cudaGraphExecDestroy(G.exec);
    G.exec = nullptr;
    G.prof_pairs.clear();
  }
  for (cudaEvent_t e : h->gprof_ev) cudaEventDestroy(e);
  h->gprof_ev.clear();
}

int ccm_set_smo2_blocks(ccm_handle* h, int block, int overlap) {
  if (!h || block < 8 || block > 128 || overlap < 0 || overlap > 64) return CCM_EINVAL;
  if (cudaDeviceSynchronize() != cudaSuccess) return CCM_ECUDA;
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device);
  for (ccm_handle* t : {h, h->adj}) {
    if (!t) continue;
    drop_graphs(t);
    const int nl = (int)t->H.levels.size();
    for (int m = 0; m + 1 < nl; ++m) {
      HostLevel& hl = t->H.levels[m];
      if (hl.n2 == 0 || hl.n2 <= t->par.ras_exact) continue;
      std::string err;
      int rc = build_smo2_blocks(hl, block, overlap, t->par.nthreads, err);
      if (!rc) rc = upload_blocks(t, m);
      if (rc) return rc;
      configure_sweep(t, t->L[m], nsm);
    }
    t->par.ras_block = block;
    t->par.ras_overlap = overlap;
    t->info.device_bytes = t->arena.bytes;
  }
  return cudaDeviceSynchronize() == cudaSuccess ? CCM_OK : CCM_ECUDA;
}

int ccm_set_launch_cap(ccm_handle* h, int max_ctas) {
  if (!h || max_ctas < 0) return CCM_EINVAL;
  if (cudaDeviceSynchronize() != cudaSuccess) return CCM_ECUDA;
  drop_graphs(h);
  h->launch_cap = max_ctas;
  if (h->adj) {
    drop_graphs(h->adj);
    h->adj->launch_cap = max_ctas;
  }
  return CCM_OK;
}

int ccm_level_launch(const ccm_handle* h, int level, int precision, int nrhs, ccm_launch_info* out) {
  if (!h || !out || level < 0 || level >= (int)h->L.size() || nrhs < 1 ||
      (precision != CCM_FP64 && precision != CCM_MIXED))
    return CCM_EINVAL;
  const int k = precision == CCM_FP64 ? 0 : 1;
  const DevLevel& L = h->L[level];
  const bool last = level == (int)h->L.size() - 1;
  const bool bj = h->par.smoother == 1 && h->par.ras_passes <= 1 && h->persistent;
  *out = ccm_launch_info{};
  if (!last && bj && L.smooth_ok[k]) {
    out->sweep_items = L.nblk + L.ntiles64;
    out->sweep_blocks = L.nblk;
    out->sweep_ctas = persistent_ctas(L.smooth_grid[k], L.smooth_cap[k], nrhs, h->launch_cap);
  }
  const HostLevel& hl = h->H.levels[level];
  for (int b = 0; b < L.nblk; ++b)
    out->block_inv_entries += (int64_t)(hl.blk[4 * b + 1] - hl.blk[4 * b]) * (hl.blk[4 * b + 3] - hl.blk[4 * b + 2]);
  if (!last && bj && L.tma && L.ntiles64r && L.restrict_ok[k]) {
    out->restrict_items = L.ntiles64r;
    out->restrict_ctas = persistent_ctas(L.restrict_grid[k], L.restrict_cap[k], nrhs, h->launch_cap);
  }
  return CCM_OK;
}

int ccm_set_cycle_params(ccm_handle* h, double omega, int nu1, int nu2, int inner_cycles, int cycle) {
  if (!h || !(omega > 0 && omega <= 1.5) || nu1 < 0 || nu2 < 0 || nu1 + nu2 < 1 || nu1 > 16 || nu2 > 16 ||
      inner_cycles < 1 || inner_cycles > 16 || cycle < 0 || cycle > 1)
    return CCM_EINVAL;
  if (cudaDeviceSynchronize() != cudaSuccess) return CCM_ECUDA;
  drop_graphs(h);
  if (h->adj) drop_graphs(h->adj);
  for (ccm_handle* t : {h, h->adj}) {
    if (!t) continue;
    const double w22 = t->S64.omega_d != 0 ? t->par.omega / t->S64.omega_d : 0.0;   // the stencil's diagonal
    t->par.omega = omega;
    t->par.nu1 = nu1;
    t->par.nu2 = nu2;
    t->par.inner_cycles = inner_cycles;
    t->par.cycle = cycle;
    if (w22 != 0) {
      t->S64.omega_d = omega / w22;
      t->S32.omega_d = (float)(omega / w22);
    }
  }
  return CCM_OK;
}

}  // extern "C"

// CCM_LOG=1 in the environment: the solves print their residual history to stderr
static bool log_enabled() {
  static const bool on = [] {
    const char* v = std::getenv("CCM_LOG");
    return v && v[0] && v[0] != '0';
  }();
  return on;
}

// r_hat = h^2 (f - N g) and the initial guess into slots [0, nb) of the level-0 FP64 arrays,
// from right-hand sides [k0, k0 + nb) of the caller's arrays (g may be NULL: g = 0).  The
// packing visits the active 32 x 8 tiles only.  ||r_hat|| of slot b goes to dnorm[B + b].
static int load_rhs(ccm_handle* h, const double* f, const double* g, const double* u, int k0, int nb, double* U0,
                    cudaStream_t s) {
  DevLevel& L = h->L[0];
  const long nu = (long)L.nx * L.ny, np = L.npad;
  const dim3 tb(dev::TX, dev::TY);
  CCM_CUDA(cudaMemsetAsync(h->rhat, 0, nb * np * sizeof(double), s));
  CCM_CUDA(cudaMemsetAsync(U0, 0, nb * np * sizeof(double), s));
  for (int b = 0; b < nb && L.ntiles; ++b) {
    const long k = k0 + b;
    KL(dev::k_pack_tiles<double, double><<<L.ntiles, tb, 0, s>>>(L.tiles, L.nx, L.ny, L.pitch, L.cls, f + k * nu,
                                                                 h->rhat + b * np, L.h * L.h));
    if (g && L.n2)
      KL(dev::k_sub_boundary<<<ceil_div(L.n2, 128), 128, 0, s>>>(L.n2, L.irr_cell, L.nb, L.seg,
                                                             g + k * h->info.n_segments, h->rhat + b * np));
    KL(dev::k_pack_tiles<double, double><<<L.ntiles, tb, 0, s>>>(L.tiles, L.nx, L.ny, L.pitch, L.cls, u + k * nu,
                                                                 U0 + b * np, 1.0));
  }
  if (h->par.precision == CCM_FP64) CCM_CUDA(cudaMemcpyAsync(L.r64, h->rhat, np * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CCM_CUDA(cudaMemsetAsync(h->dnorm + h->B, 0, nb * sizeof(unsigned long long), s));
  if (L.ntiles)
    KL(launch_k(dev::k_absmax_tiles<double>, dim3(std::min(L.ntiles, 1216), nb), tb, 0, s, L.tiles, L.ntiles, L.nx, L.ny,
                L.pitch, L.cls, (const double*)h->rhat, h->dnorm + h->B, np));
  return CCM_OK;
}

// max |r_hat - L U0| of one right-hand side into dnorm[0] (no host synchronisation)
static void initial_residual(ccm_handle* h, const double* U0, cudaStream_t s) {
  DevLevel& L = h->L[0];
  if (h->par.precision != CCM_FP64 && h->fused_outer) {
    outer_residual32(h, s);
    return;
  }
  launch_regular<double>(h, L, U0, h->rhat, L.t64, true, s);
  if (L.n2)
    KL(launch_k(dev::k_rows<double, double, true, true>, ceil_div(L.n2, 128), 128, 0, s,
        L.n2, L.W, L.irr_cell, L.ell_col, L.ell64, U0, h->rhat, L.t64, nullptr, nullptr, nullptr));
  cudaMemsetAsync(h->dnorm, 0, sizeof(unsigned long long), s);
  KL(launch_k(dev::k_absmax<double>, std::min(ceil_div(L.npad, 256), 1216), 256, 0, s, L.npad, L.cls,
              (const double*)L.t64, h->dnorm, 0L));
}

namespace {

// ccm_solve; keep_empty: the empty cells of u keep the values they had (ccm_solve_host)
int solve_impl(ccm_handle* h, const double* f, const double* g, double* u, int nrhs, void* stream, ccm_stats* st,
               bool keep_empty) {
  if (!h || !f || !u || nrhs < 1) return CCM_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  DevLevel& L = h->L[0];
  const long nu = (long)L.nx * L.ny, np = L.npad;
  dim3 pg(ceil_div(L.nx, 128), L.ny);
  const bool fp64 = h->par.precision == CCM_FP64;
  const int bmax = fp64 ? 1 : h->bmax;
  int result = CCM_OK;
  std::vector<double> rnorm(bmax), rel(bmax);
  // right-hand sides [k0, k0 + nb) advance together, in slot b of every batched array
  for (int k0 = 0; k0 < nrhs; k0 += bmax) {
    const int nb = std::min(bmax, nrhs - k0);
    h->nb = nb;
    int rc = capture_iteration(h, fp64, s);
    if (rc) {
      h->nb = 1;
      return rc;
    }
    ccm_handle::Graph& G = h->graph[fp64 ? 1 : 0];
    double* U0 = G.u0;
    rc = load_rhs(h, f, g, u, k0, nb, U0, s);
    if (rc) {
      h->nb = 1;
      return rc;
    }
    // initial residual (one right-hand side at a time outside the fused mixed form); its norms
    // and ||r_hat|| come back in one synchronisation
    initial_residual(h, U0, s);
    CCM_CUDA(cudaMemcpyAsync(h->hnorm, h->dnorm, nb * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    CCM_CUDA(cudaMemcpyAsync(h->hnorm + h->B, h->dnorm + h->B, nb * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    CCM_CUDA(cudaStreamSynchronize(s));
    for (int b = 0; b < nb; ++b) {
      std::memcpy(&rnorm[b], &h->hnorm[h->B + b], sizeof(double));
      if (rnorm[b] == 0) rnorm[b] = 1;
      std::memcpy(&rel[b], &h->hnorm[b], sizeof(double));
    }
    // the worst right-hand side of the group decides; stats report it
    auto worst = [&]() {
      double w = 0;
      for (int b = 0; b < nb; ++b) {
        const double r = rel[b] / rnorm[b];
        if (!std::isfinite(r)) return r;
        w = std::max(w, r);
      }
      return w;
    };
    double wr = worst();
    ccm_stats local{};
    local.history[0] = wr;
    int it = 0;
    while (std::isfinite(wr) && wr > h->par.rtol && it < h->par.max_iter) {
      CCM_CUDA(cudaGraphLaunch(G.exec, s));
      g_launches.fetch_add(G.launches);
      CCM_CUDA(cudaStreamSynchronize(s));
      for (int b = 0; b < nb; ++b) std::memcpy(&rel[b], &h->hnorm[b], sizeof(double));
      wr = worst();
      ++it;
      if (*h->herr) {
        result = CCM_ETIMEOUT;
        *h->herr = 0;
        cudaMemsetAsync(h->derr, 0, sizeof(int), s);
        break;
      }
      if (it < 64) local.history[it] = wr;
      for (int p : G.prof_pairs) {
        float t = 0;
        if (cudaEventElapsedTime(&t, h->gprof_ev[p], h->gprof_ev[p + 1]) == cudaSuccess) {
          h->prof_ms += t;
          h->prof_n += 1;
        }
      }
    }
    if (result == CCM_ETIMEOUT) {
    } else if (!std::isfinite(wr)) result = CCM_ENOTFINITE;
    else if (wr > h->par.rtol && result == CCM_OK) result = CCM_ENOCONV;
    // the non-empty cells over the active tiles; without keep_empty the array is cleared first
    for (int b = 0; b < nb; ++b) {
      if (!keep_empty) CCM_CUDA(cudaMemsetAsync(u + (k0 + b) * nu, 0, nu * sizeof(double), s));
      if (L.ntiles)
        KL(dev::k_unpack_tiles<double><<<L.ntiles, dim3(dev::TX, dev::TY), 0, s>>>(L.tiles, L.nx, L.ny, L.pitch, L.cls,
                                                                                 U0 + b * np, u + (k0 + b) * nu, 1.0));
    }
    local.iterations = it;
    local.rel_residual = wr;
    if (st) *st = local;
    if (log_enabled()) {
      std::fprintf(stderr, "ccm_solve: right-hand sides %d-%d, %s, %d outer iterations, status %d\n", k0,
                   k0 + nb - 1, fp64 ? "FP64" : "mixed", it, result);
      for (int j = 0; j <= std::min(it, 63); ++j)
        std::fprintf(stderr, "ccm_solve:   iteration %2d  rel. residual %.3e\n", j, local.history[j]);
    }
    if (result == CCM_ETIMEOUT) break;
  }
  h->nb = 1;
  CCM_CUDA(cudaGetLastError());
  return result;
}

}  // namespace

extern "C" {

int ccm_solve(ccm_handle* h, const double* f, const double* g, double* u, int nrhs, void* stream, ccm_stats* st) {
  return solve_impl(h, f, g, u, nrhs, stream, st, false);
}

}  // extern "C"

// ---------------------------------------------------------------- many problems, one graph

struct ccm_group {
  std::vector<ccm_handle*> m;
  std::vector<double*> u0;            // per member: the level-0 FP64 iterate its iteration updates
  std::vector<long long> launches;    // per member: kernel launches of one outer iteration
  cudaGraphExec_t exec = nullptr;
  bool pdl = true;                    // the members' launches keep their programmatic edges
  Arena arena;
  dev::GroupArgs A{};
  unsigned long long* rnorm = nullptr;   // device, per member
  int* it = nullptr;                     // device loop counter
  // pinned host copies of the per-member results
  int* h_iters = nullptr;
  int* h_failed = nullptr;
  double* h_rel = nullptr;
  double* h_hist = nullptr;
};

namespace {

// member h's outer iteration (single right-hand side) as an uninstantiated graph
int capture_member(ccm_handle* h, cudaStream_t user, cudaGraph_t* out, long long* launches, double** u0) {
  const bool fp64 = h->par.precision == CCM_FP64;
  h->nb = 1;
  if (!h->cap_stream) CCM_CUDA(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  CCM_CUDA(cudaStreamSynchronize(user));
  cudaStream_t s = h->cap_stream;
  const int cur64 = h->L[0].cur64;
  const int prof = h->prof_class;
  h->prof_class = 0;                  // no event nodes: conditional bodies cannot hold them
  CCM_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  h->capturing = true;
  const long long l0 = g_launches.load();
  iteration_body(h, fp64, s, false);
  *launches = g_launches.load() - l0;
  g_launches.fetch_sub(*launches);
  h->capturing = false;
  h->prof_class = prof;
  cudaError_t e = cudaStreamEndCapture(s, out);
  h->L[0].cur64 = cur64;
  *u0 = fp64 ? h->L[0].u64[cur64] : h->uhat;
  return e == cudaSuccess ? CCM_OK : CCM_ECUDA;
}

// WHILE(any member active) { IF(member k active) { iteration of k } for every k; decide }
int build_group_graph(ccm_group* G, cudaStream_t user) {
  const int n = (int)G->m.size();
  std::vector<cudaGraph_t> body(n, nullptr);
  G->u0.assign(n, nullptr);
  G->launches.assign(n, 0);
  const bool pdl0 = t_pdl;
  t_pdl = G->pdl;
  int rc = CCM_OK;
  for (int k = 0; k < n && rc == CCM_OK; ++k) rc = capture_member(G->m[k], user, &body[k], &G->launches[k], &G->u0[k]);
  t_pdl = pdl0;
  cudaGraph_t graph = nullptr;
  auto done = [&](int r) {
    for (cudaGraph_t b : body)
      if (b) cudaGraphDestroy(b);
    if (graph) cudaGraphDestroy(graph);
    return r;
  };
  if (rc) return done(rc);
  if (cudaGraphCreate(&graph, 0) != cudaSuccess) return done(CCM_ECUDA);
  // every condition starts each launch at 0 (nothing runs) until k_group_init sets it
  cudaGraphConditionalHandle hw;
  std::vector<cudaGraphConditionalHandle> hk(n);
  if (cudaGraphConditionalHandleCreate(&hw, graph, 0, cudaGraphCondAssignDefault) != cudaSuccess) return done(CCM_ECUDA);
  for (int k = 0; k < n; ++k)
    if (cudaGraphConditionalHandleCreate(&hk[k], graph, 0, cudaGraphCondAssignDefault) != cudaSuccess)
      return done(CCM_ECUDA);
  G->A.hw = hw;
  if (cudaMemcpy((void*)G->A.hk, hk.data(), n * sizeof(cudaGraphConditionalHandle), cudaMemcpyHostToDevice) != cudaSuccess)
    return done(CCM_ECUDA);
  dev::GroupArgs args = G->A;
  void* kargs[] = {&args};
  cudaKernelNodeParams kp{};
  kp.func = (void*)dev::k_group_init;
  kp.gridDim = dim3(1);
  kp.blockDim = dim3(256);
  kp.kernelParams = kargs;
  cudaGraphNode_t init, loop, decide;
  if (cudaGraphAddKernelNode(&init, graph, nullptr, 0, &kp) != cudaSuccess) return done(CCM_ECUDA);
  cudaGraphNodeParams wp{};
  wp.type = cudaGraphNodeTypeConditional;
  wp.conditional.handle = hw;
  wp.conditional.type = cudaGraphCondTypeWhile;
  wp.conditional.size = 1;
  if (cudaGraphAddNode(&loop, graph, &init, nullptr, 1, &wp) != cudaSuccess) return done(CCM_ECUDA);
  cudaGraph_t lbody = wp.conditional.phGraph_out[0];
  std::vector<cudaGraphNode_t> ifs(n);
  for (int k = 0; k < n; ++k) {
    cudaGraphNodeParams ip{};
    ip.type = cudaGraphNodeTypeConditional;
    ip.conditional.handle = hk[k];
    ip.conditional.type = cudaGraphCondTypeIf;
    ip.conditional.size = 1;
    if (cudaGraphAddNode(&ifs[k], lbody, nullptr, nullptr, 0, &ip) != cudaSuccess) return done(CCM_ECUDA);
    cudaGraphNode_t child;
    if (cudaGraphAddChildGraphNode(&child, ip.conditional.phGraph_out[0], nullptr, 0, body[k]) != cudaSuccess)
      return done(CCM_ECUDA);
  }
  kp.func = (void*)dev::k_group_decide;
  if (cudaGraphAddKernelNode(&decide, lbody, ifs.data(), n, &kp) != cudaSuccess) return done(CCM_ECUDA);
  if (cudaGraphInstantiate(&G->exec, graph, 0) != cudaSuccess) {
    G->exec = nullptr;
    cudaGetLastError();
    return done(CCM_ECUDA);
  }
  return done(CCM_OK);
}

}  // namespace

extern "C" {

int ccm_group_create(ccm_handle* const* members, int count, void* stream, ccm_group** out) {
  if (!members || count < 1 || !out) return CCM_EINVAL;
  *out = nullptr;
  for (int k = 0; k < count; ++k) {
    if (!members[k]) return CCM_EINVAL;
    for (int j = 0; j < k; ++j)
      if (members[j] == members[k]) return CCM_EINVAL;     // one slot of state per handle
  }
  cudaStream_t s = (cudaStream_t)stream;
  std::unique_ptr<ccm_group> G(new ccm_group());
  G->m.assign(members, members + count);
  Arena& A = G->arena;
  const int n = count;
  std::vector<const unsigned long long*> norms(n);
  std::vector<const int*> errs(n);
  std::vector<double> rtol(n);
  std::vector<int> maxit(n);
  for (int k = 0; k < n; ++k) {
    norms[k] = G->m[k]->dnorm;
    errs[k] = G->m[k]->derr;
    rtol[k] = G->m[k]->par.rtol;
    maxit[k] = G->m[k]->par.max_iter;
  }
  dev::GroupArgs& a = G->A;
  a.n = n;
  a.norm = A.upload(norms);
  a.err = A.upload(errs);
  a.rtol = A.upload(rtol);
  a.max_iter = A.upload(maxit);
  a.hk = A.alloc<cudaGraphConditionalHandle>(n);
  G->rnorm = A.alloc<unsigned long long>(n);
  a.rnorm = G->rnorm;
  a.act = A.alloc<int>(n);
  a.iters = A.alloc<int>(n);
  a.failed = A.alloc<int>(n);
  a.rel = A.alloc<double>(n);
  a.hist = A.alloc<double>((long)n * dev::GROUP_HIST);
  G->it = A.alloc<int>(1);
  a.it = G->it;
  if (A.err != cudaSuccess) return A.err == cudaErrorMemoryAllocation ? CCM_ENOMEM : CCM_ECUDA;
  if (cudaMallocHost(&G->h_iters, n * sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&G->h_failed, n * sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&G->h_rel, n * sizeof(double)) != cudaSuccess ||
      cudaMallocHost(&G->h_hist, (long)n * dev::GROUP_HIST * sizeof(double)) != cudaSuccess) {
    ccm_group_free(G.release());
    return CCM_ENOMEM;
  }
  int rc = build_group_graph(G.get(), s);
  if (rc == CCM_ECUDA) {
    // a runtime that rejects programmatic edges inside conditional bodies: plain edges
    G->pdl = false;
    rc = build_group_graph(G.get(), s);
  }
  if (rc) {
    ccm_group_free(G.release());
    return rc;
  }
  *out = G.release();
  return CCM_OK;
}

int ccm_group_solve(ccm_group* G, const double* const* f, const double* const* g, double* const* u, void* stream,
                    ccm_stats* st) {
  if (!G || !f || !u) return CCM_EINVAL;
  const int n = (int)G->m.size();
  for (int k = 0; k < n; ++k)
    if (!f[k] || !u[k]) return CCM_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  // right-hand sides, initial guesses, ||r_hat|| and the initial residual of every member
  for (int k = 0; k < n; ++k) {
    ccm_handle* h = G->m[k];
    h->nb = 1;
    int rc = load_rhs(h, f[k], g ? g[k] : nullptr, u[k], 0, 1, G->u0[k], s);
    if (rc) return rc;
    CCM_CUDA(cudaMemcpyAsync(G->rnorm + k, h->dnorm + h->B, sizeof(unsigned long long), cudaMemcpyDeviceToDevice, s));
    initial_residual(h, G->u0[k], s);
  }
  CCM_CUDA(cudaGraphLaunch(G->exec, s));
  CCM_CUDA(cudaMemcpyAsync(G->h_iters, G->A.iters, n * sizeof(int), cudaMemcpyDeviceToHost, s));
  CCM_CUDA(cudaMemcpyAsync(G->h_failed, G->A.failed, n * sizeof(int), cudaMemcpyDeviceToHost, s));
  CCM_CUDA(cudaMemcpyAsync(G->h_rel, G->A.rel, n * sizeof(double), cudaMemcpyDeviceToHost, s));
  CCM_CUDA(cudaMemcpyAsync(G->h_hist, G->A.hist, (long)n * dev::GROUP_HIST * sizeof(double), cudaMemcpyDeviceToHost, s));
  int result = CCM_OK;
  for (int k = 0; k < n; ++k) {
    ccm_handle* h = G->m[k];
    DevLevel& L = h->L[0];
    dim3 pg(ceil_div(L.nx, 128), L.ny);
    KL(dev::k_unpack<double><<<pg, 128, 0, s>>>(L.nx, L.ny, L.pitch, L.cls, G->u0[k], u[k], 1.0));
  }
  CCM_CUDA(cudaStreamSynchronize(s));
  long long total = 2;   // k_group_init and the last k_group_decide
  int loops = 0;
  for (int k = 0; k < n; ++k) {
    ccm_handle* h = G->m[k];
    const int it = G->h_iters[k];
    const double r = G->h_rel[k];
    total += (long long)it * G->launches[k];
    loops = std::max(loops, it);
    int rk = CCM_OK;
    if (G->h_failed[k]) {
      rk = CCM_ETIMEOUT;
      cudaMemsetAsync(h->derr, 0, sizeof(int), s);
    } else if (!std::isfinite(r)) {
      rk = CCM_ENOTFINITE;
    } else if (r > h->par.rtol) {
      rk = CCM_ENOCONV;
    }
    if (result == CCM_OK) result = rk;
    if (log_enabled())
      std::fprintf(stderr, "ccm_group_solve: member %d, %d outer iterations, rel. residual %.3e, status %d\n", k, it,
                   r, rk);
    if (st) {
      ccm_stats& o = st[k];
      o = ccm_stats{};
      o.iterations = it;
      o.rel_residual = r;
      for (int j = 0; j <= std::min(it, dev::GROUP_HIST - 1); ++j) o.history[j] = G->h_hist[(long)k * dev::GROUP_HIST + j];
    }
  }
  g_launches.fetch_add(total + std::max(0, loops - 1));
  CCM_CUDA(cudaGetLastError());
  return result;
}

int ccm_group_query(const ccm_group* G, int* members, int* programmatic) {
  if (!G) return CCM_EINVAL;
  if (members) *members = (int)G->m.size();
  if (programmatic) *programmatic = G->pdl ? 1 : 0;
  return CCM_OK;
}

void ccm_group_free(ccm_group* G) {
  if (!G) return;
  cudaDeviceSynchronize();
  if (G->exec) cudaGraphExecDestroy(G->exec);
  G->arena.release();
  if (G->h_iters) cudaFreeHost(G->h_iters);
  if (G->h_failed) cudaFreeHost(G->h_failed);
  if (G->h_rel) cudaFreeHost(G->h_rel);
  if (G->h_hist) cudaFreeHost(G->h_hist);
  delete G;
}

}  // extern "C"

namespace {

// a pointer the kernels can dereference for `bytes` bytes: device or managed memory and
// pinned host memory as they are (pinned host memory through its device address: the GPU
// reads and writes it over the host link, with no copy), pageable host memory as it is where
// the device reads pageable memory coherently (Grace's address translation), else a device
// staging buffer (copied in, and copied back by stage_back)
struct HostView {
  void* dev = nullptr;
  void* staged = nullptr;
  const void* host = nullptr;
  size_t bytes = 0;
};

int host_view(const void* p, size_t bytes, bool read, cudaStream_t s, HostView& v) {
  v = HostView{};
  v.host = p;
  v.bytes = bytes;
  if (!p) return CCM_OK;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    at.type = cudaMemoryTypeUnregistered;
  }
  if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) {
    v.dev = const_cast<void*>(p);
    return CCM_OK;
  }
  if (at.type == cudaMemoryTypeHost && at.devicePointer) {
    v.dev = at.devicePointer;
    return CCM_OK;
  }
  int dev = 0, pageable = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, dev);
  if (pageable) {
    v.dev = const_cast<void*>(p);
    return CCM_OK;
  }
  if (cudaMalloc(&v.staged, bytes) != cudaSuccess) return CCM_ENOMEM;
  v.dev = v.staged;
  if (read && cudaMemcpyAsync(v.staged, p, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) return CCM_ECUDA;
  return CCM_OK;
}

int stage_back(HostView& v, cudaStream_t s) {
  if (!v.staged) return CCM_OK;
  if (cudaMemcpyAsync(const_cast<void*>(v.host), v.staged, v.bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return CCM_ECUDA;
  return CCM_OK;
}

void release(HostView& v) {
  if (v.staged) cudaFree(v.staged);
  v.staged = nullptr;
}

}  // namespace

extern "C" {

int ccm_solve_host(ccm_handle* h, const double* f, const double* g, double* u, int nrhs, void* stream,
                   ccm_stats* st) {
  if (!h || !f || !u || nrhs < 1) return CCM_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t cells = (size_t)h->L[0].nx * h->L[0].ny * nrhs;
  HostView vf, vg, vu;
  int rc = host_view(f, cells * sizeof(double), true, s, vf);
  if (!rc) rc = host_view(g, (size_t)h->info.n_segments * nrhs * sizeof(double), true, s, vg);
  if (!rc) rc = host_view(u, cells * sizeof(double), true, s, vu);
  if (!rc) {
    rc = solve_impl(h, (const double*)vf.dev, (const double*)vg.dev, (double*)vu.dev, nrhs, stream, st, true);
    // the solution in u (also after CCM_ENOCONV, where u holds the last iterate)
    const int rb = stage_back(vu, s);
    if (rc == CCM_OK || rc == CCM_ENOCONV) rc = rc ? rc : rb;
    if (!vu.staged && cudaStreamSynchronize(s) != cudaSuccess && rc == CCM_OK) rc = CCM_ECUDA;
  }
  release(vf);
  release(vg);
  release(vu);
  return rc;
}

int ccm_solve_T(ccm_handle* h, const double* rhs, double* lambda, int nrhs, void* stream, ccm_stats* st) {
  if (!h || !rhs || !lambda || nrhs < 1) return CCM_EINVAL;
  if (!h->adj) {
    std::unique_ptr<ccm_handle> t(new ccm_handle());
    t->par = h->par;
    t->a = h->a;
    t->b = h->b;
    t->c = h->c;
    t->cross = h->cross;
    t->device = h->device;
    std::string err;
    int rc;
    try {
      rc = build_transposed(h->H, h->par, t->H, err);
    } catch (const std::bad_alloc&) {
      return CCM_ENOMEM;
    }
    if (rc) return rc;
    rc = upload_hierarchy(t.get());
    if (rc) return rc;
    t->info = h->info;
    t->info.n_segments = 0;
    h->adj = t.release();
  }
  return ccm_solve(h->adj, rhs, nullptr, lambda, nrhs, stream, st);
}

// ---- level components

int ccm_level_apply(ccm_handle* h, int level, const double* u, double* out, void* stream) {
  if (check_level(h, level) || !u || !out) return CCM_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  DevLevel& L = h->L[level];
  dim3 pg(ceil_div(L.nx, 128), L.ny);
  KL(dev::k_pack<double, double><<<pg, 128, 0, s>>>(L.nx, L.ny, L.pitch, L.cls, u, L.t64, 1.0));
  launch_regular<double>(h, L, L.t64, nullptr, L.r64, false, s);
  if (L.n2)
    KL(launch_k(dev::k_rows<double, double, false, true>, ceil_div(L.n2, 128), 128, 0, s, 
        L.n2, L.W, L.irr_cell, L.ell_col, L.ell64, L.t64, nullptr, L.r64, L.nb, L.seg, nullptr));
  KL(dev::k_unpack<double><<<pg, 128, 0, s>>>(L.nx, L.ny, L.pitch, L.cls, L.r64, out, 1.0 / (L.h * L.h)));
  CCM_CUDA(cudaGetLastError());
  return CCM_OK;
}

int ccm_level_smooth(ccm_handle* h, int level, double* u, const double* r, int precision, void* stream) {
  if (check_level(h, level) || !u || !r || level == (int)h->L.size() - 1) return CCM_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  DevLevel& L = h->L[level];
  dim3 pg(ceil_div(L.nx, 128), L.ny);
  if (precision == CCM_FP64) {
    load_level<double>(h, L, u, r, s);
    smooth_step<double>(h, L, s);
    KL(dev::k_unpack<double><<<pg, 128, 0, s>>>(L.nx, L.ny, L.pitch, L.cls, U<double>(L), u, 1.0));
  } else {
    load_level<float>(h, L, u, r, s);
    smooth_step<float>(h, L, s);
    KL(dev::k_unpack<float><<<pg, 128, 0, s>>>(L.nx, L.ny, L.pitch, L.cls, U<float>(L), u, 1.0));
  }
  CCM_CUDA(cudaGetLastError());
  return CCM_OK;
}

int ccm_level_restrict(ccm_handle* h, int level, const double* u, const double* r, double* rc, void* stream) {
  if (check_level(h, level) || level == (int)h->L.size() - 1 || !u || !r || !rc) return CCM_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  DevLevel& F = h->L[level];
  DevLevel& C = h->L[level + 1];
  load_level<double>(h, F, u, r, s);
  cudaMemsetAsync(C.r64, 0, C.npad * sizeof(double), s);
  restrict_to<double>(h, F, C, s);
  dim3 pg(ceil_div(C.nx, 128), C.ny);
  KL(dev::k_unpack<double><<<pg, 128, 0, s>>>(C.nx, C.ny, C.pitch, C.cls, C.r64, rc, 1.0 / (C.h * C.h)));
  CCM_CUDA(cudaGetLastError());
  return CCM_OK;
}

int ccm_level_prolong(ccm_handle* h, int level, const double* uc, double* u, void* stream) {
  if (check_level(h, level) || level == (int)h->L.size() - 1 || !u || !uc) return CCM_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  DevLevel& F = h->L[level];
  DevLevel& C = h->L[level + 1];
  load_level<double>(h, F, u, nullptr, s);
  load_level<double>(h, C, uc, nullptr, s);
  prolong_from<double>(h, F, C, s);
  dim3 pg(ceil_div(F.nx, 128), F.ny);
  KL(dev::k_unpack<double><<<pg, 128, 0, s>>>(F.nx, F.ny, F.pitch, F.cls, U<double>(F), u, 1.0));
  CCM_CUDA(cudaGetLastError());
  return CCM_OK;
}

int ccm_level_prolong_smooth(ccm_handle* h, int level, double* u, const double* uc, const double* r, int precision,
                             void* stream) {
  if (check_level(h, level) || level == (int)h->L.size() - 1 || !u || !uc || !r) return CCM_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  DevLevel& F = h->L[level];
  DevLevel& C = h->L[level + 1];
  dim3 pg(ceil_div(F.nx, 128), F.ny);
  if (precision == CCM_FP64) {
    load_level<double>(h, F, u, r, s);
    load_level<double>(h, C, uc, nullptr, s);
    smooth_step<double>(h, F, s, U<double>(C), C.pitch);
    KL(dev::k_unpack<double><<<pg, 128, 0, s>>>(F.nx, F.ny, F.pitch, F.cls, U<double>(F), u, 1.0));
  } else {
    load_level<float>(h, F, u, r, s);
    load_level<float>(h, C, uc, nullptr, s);
    smooth_step<float>(h, F, s, U<float>(C), C.pitch);
    KL(dev::k_unpack<float><<<pg, 128, 0, s>>>(F.nx, F.ny, F.pitch, F.cls, U<float>(F), u, 1.0));
  }
  CCM_CUDA(cudaGetLastError());
  return CCM_OK;
}

int ccm_bottom_solve(ccm_handle* h, const double* r, double* u, void* stream) {
  if (!h || !r || !u) return CCM_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  DevLevel& B = h->L.back();
  load_level<double>(h, B, nullptr, r, s);
  bottom<double>(h, B, s);
  dim3 pg(ceil_div(B.nx, 128), B.ny);
  KL(dev::k_unpack<double><<<pg, 128, 0, s>>>(B.nx, B.ny, B.pitch, B.cls, U<double>(B), u, 1.0));
  CCM_CUDA(cudaGetLastError());
  return CCM_OK;
}

int ccm_vcycle(ccm_handle* h, double* u, const double* r, int precision, void* stream) {
  if (!h || !u || !r) return CCM_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  DevLevel& L = h->L[0];
  dim3 pg(ceil_div(L.nx, 128), L.ny);
  if (precision == CCM_FP64) {
    load_level<double>(h, L, u, r, s);
    vcycle<double>(h, 0, s);
    KL(dev::k_unpack<double><<<pg, 128, 0, s>>>(L.nx, L.ny, L.pitch, L.cls, U<double>(L), u, 1.0));
  } else {
    load_level<float>(h, L, u, r, s);
    vcycle<float>(h, 0, s);
    KL(dev::k_unpack<float><<<pg, 128, 0, s>>>(L.nx, L.ny, L.pitch, L.cls, U<float>(L), u, 1.0));
  }
  CCM_CUDA(cudaGetLastError());
  return CCM_OK;
}

int ccm_fmg(ccm_handle* h, double* u, const double* r, int precision, void* stream) {
  if (!h || !u || !r) return CCM_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  DevLevel& L = h->L[0];
  dim3 pg(ceil_div(L.nx, 128), L.ny);
  if (precision == CCM_FP64) {
    load_level<double>(h, L, u, r, s);
    fmg<double>(h, s);
    KL(dev::k_unpack<double><<<pg, 128, 0, s>>>(L.nx, L.ny, L.pitch, L.cls, U<double>(L), u, 1.0));
  } else {
    load_level<float>(h, L, u, r, s);
    fmg<float>(h, s);
    KL(dev::k_unpack<float><<<pg, 128, 0, s>>>(L.nx, L.ny, L.pitch, L.cls, U<float>(L), u, 1.0));
  }
  CCM_CUDA(cudaGetLastError());
  return CCM_OK;
}

int64_t ccm_launch_count(void) { return (int64_t)g_launches.load(); }

}  // extern "C"

namespace {

// self-test of the bounded wait: one CTA waits, through the tile-wait helper of the solve
// kernels, on an mbarrier phase that nothing completes (no copy is issued, nobody arrives), so
// the wait runs out, sets the error word and the kernel returns
__global__ void k_wait_selftest(int* err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) dev::mbar_init(&bar, 1);
  __syncthreads();
  dev::tile_wait(&bar, err);
}

}  // namespace

extern "C" {

int ccm_wait_selftest(ccm_handle* h, void* stream) {
  if (!h) return CCM_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  KL(k_wait_selftest<<<1, 32, 0, s>>>(h->derr));
  CCM_CUDA(cudaMemcpyAsync(h->herr, h->derr, sizeof(int), cudaMemcpyDeviceToHost, s));
  CCM_CUDA(cudaStreamSynchronize(s));
  const int timed_out = *h->herr;
  *h->herr = 0;
  CCM_CUDA(cudaMemsetAsync(h->derr, 0, sizeof(int), s));
  CCM_CUDA(cudaStreamSynchronize(s));
  return timed_out ? CCM_ETIMEOUT : CCM_OK;
}

int ccm_profile(ccm_handle* h, int kernel_class) {
  if (!h || kernel_class < 0 || kernel_class > CCM_PROF_RESTRICT_FP32) return CCM_EINVAL;
  if (kernel_class != h->prof_class) {
    cudaDeviceSynchronize();
    drop_graphs(h);
  }
  h->prof_class = kernel_class;
  h->prof_used = 0;
  h->prof_ms = 0;
  h->prof_n = 0;
  return CCM_OK;
}

int ccm_profile_read(ccm_handle* h, double* ms, int64_t* launches) {
  if (!h || !ms || !launches) return CCM_EINVAL;
  double tot = 0;
  for (int k = 0; k + 1 < h->prof_used; k += 2) {
    CCM_CUDA(cudaEventSynchronize(h->prof_ev[k + 1]));
    float t = 0;
    CCM_CUDA(cudaEventElapsedTime(&t, h->prof_ev[k], h->prof_ev[k + 1]));
    tot += t;
  }
  *ms = tot + h->prof_ms;
  *launches = h->prof_used / 2 + h->prof_n;
  h->prof_used = 0;
  h->prof_ms = 0;
  h->prof_n = 0;
  return CCM_OK;
}

void ccm_free(ccm_handle* h) {
  if (!h) return;
  if (h->adj) ccm_free(h->adj);
  cudaDeviceSynchronize();
  drop_graphs(h);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  for (cudaEvent_t e : h->prof_ev) cudaEventDestroy(e);
  h->arena.release();
  if (h->hnorm) cudaFreeHost(h->hnorm);
  if (h->herr) cudaFreeHost(h->herr);
  delete h;
}

}  // extern "C"
