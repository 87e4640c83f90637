// The setup's batched fits on the GPU (FitBatcher of host.h): the level's cut-cell moments,
// volumes and boundary-piece moments go to the device once per call, the (row, candidate)
// pairs as index lists, and k_plg_fit / k_plg_cond return the coefficients, the weighted
// norms and the condition numbers.  Blocking; device memory is released before returning.
#include <cstring>
#include <memory>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "host.h"
#include "plgfit.cuh"

namespace ccm {
namespace {

// device buffers released at scope exit
struct DevBufs {
  std::vector<void*> p;
  cudaError_t err = cudaSuccess;
  template <typename T>
  T* put(const std::vector<T>& v) {
    if (err != cudaSuccess) return nullptr;
    void* d = nullptr;
    const size_t n = std::max<size_t>(1, v.size()) * sizeof(T);
    err = cudaMalloc(&d, n);
    if (err != cudaSuccess) return nullptr;
    p.push_back(d);
    if (!v.empty()) err = cudaMemcpy(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
    return (T*)d;
  }
  template <typename T>
  T* get(size_t n) {
    if (err != cudaSuccess) return nullptr;
    void* d = nullptr;
    err = cudaMalloc(&d, std::max<size_t>(1, n) * sizeof(T));
    if (err != cudaSuccess) return nullptr;
    p.push_back(d);
    return (T*)d;
  }
  ~DevBufs() {
    for (void* d : p) cudaFree(d);
  }
};

struct LevelTables {
  std::unordered_map<int, int> id;      // cut cell -> moment id
  std::vector<double> mom, vol, seg_mom, seg_gamma;
  std::vector<int32_t> seg_bc;
};

void level_tables(const CutLevel& cg, LevelTables& T) {
  T.id.reserve(cg.mom.size() * 2);
  for (const auto& kv : cg.mom) {
    const int id = (int)T.vol.size();
    T.id[kv.first] = id;
    T.mom.insert(T.mom.end(), kv.second.begin(), kv.second.end());
    T.vol.push_back(cg.vol[kv.first]);
  }
  const size_t ns = cg.segs.size();
  T.seg_bc.assign(cg.seg_bc.begin(), cg.seg_bc.end());
  T.seg_mom.resize(ns * 3 * NMOM);
  T.seg_gamma.resize(ns * 2);
  for (size_t s = 0; s < ns; ++s) {
    for (int k = 0; k < NMOM; ++k) {
      T.seg_mom[(s * 3 + 0) * NMOM + k] = cg.bm0[s][k];
      T.seg_mom[(s * 3 + 1) * NMOM + k] = cg.bmx[s][k];
      T.seg_mom[(s * 3 + 2) * NMOM + k] = cg.bmy[s][k];
    }
    T.seg_gamma[2 * s] = cg.seg_gamma[s][0];
    T.seg_gamma[2 * s + 1] = cg.seg_gamma[s][1];
  }
}

int mom_id(const LevelTables& T, int lin) {
  auto it = T.id.find(lin);
  return it == T.id.end() ? -1 : it->second;
}

class DeviceFitter final : public FitBatcher {
 public:
  int fit(const CutLevel& cg, double a, double b, double c, const std::vector<int32_t>& row_cell,
          const std::vector<std::array<int, 15>>& cand, std::vector<double>& beta, std::vector<double>& norm,
          std::vector<uint8_t>& ok) override {
    return run(cg, a, b, c, row_cell, cand, &beta, &norm, &ok, nullptr);
  }
  int cond(const CutLevel& cg, const std::vector<int32_t>& row_cell, const std::vector<std::array<int, 15>>& cand,
           std::vector<double>& cond) override {
    return run(cg, 0, 0, 0, row_cell, cand, nullptr, nullptr, nullptr, &cond);
  }

 private:
  int run(const CutLevel& cg, double a, double b, double c, const std::vector<int32_t>& row_cell,
          const std::vector<std::array<int, 15>>& cand, std::vector<double>* beta, std::vector<double>* norm,
          std::vector<uint8_t>* ok, std::vector<double>* cond) {
    const size_t n = cand.size();
    if (n == 0) {
      if (beta) beta->clear();
      if (norm) norm->clear();
      if (ok) ok->clear();
      if (cond) cond->clear();
      return CCM_OK;
    }
    LevelTables T;
    level_tables(cg, T);
    std::vector<int32_t> rw(4 * n), cells(30 * n);
    for (size_t k = 0; k < n; ++k) {
      const int lin = row_cell[k];
      rw[4 * k] = lin % cg.nx;
      rw[4 * k + 1] = lin / cg.nx;
      rw[4 * k + 2] = mom_id(T, lin);
      auto sit = cg.seg_of.find(lin);
      rw[4 * k + 3] = sit == cg.seg_of.end() ? -1 : sit->second;
      for (int q = 0; q < 15; ++q) {
        cells[30 * k + 2 * q] = cand[k][q];
        cells[30 * k + 2 * q + 1] = mom_id(T, cand[k][q]);
      }
    }
    DevBufs D;
    dev::FitLevel L{};
    L.nx = cg.nx;
    L.h = cg.h;
    L.a = a;
    L.b = b;
    L.c = c;
    L.mom = D.put(T.mom);
    L.vol = D.put(T.vol);
    L.seg_bc = D.put(T.seg_bc);
    L.seg_mom = D.put(T.seg_mom);
    L.seg_gamma = D.put(T.seg_gamma);
    const Mom& pm = pure_moments();
    for (int k = 0; k < NMOM; ++k) L.pure[k] = pm[k];
    dev::FitBatch B{};
    B.n = (int)n;
    B.row = D.put(rw);
    B.cells = D.put(cells);
    if (cond) {
      B.cond = D.get<double>(n);
    } else {
      B.beta = D.get<double>(16 * n);
      B.norm = D.get<double>(n);
      B.ok = D.get<uint8_t>(n);
    }
    if (D.err != cudaSuccess) return D.err == cudaErrorMemoryAllocation ? CCM_ENOMEM : CCM_ECUDA;
    const unsigned grid = (unsigned)((n + 3) / 4);
    if (cond) dev::k_plg_cond<<<grid, 128>>>(L, B);
    else dev::k_plg_fit<<<grid, 128>>>(L, B);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return CCM_ECUDA;
    if (cond) {
      cond->resize(n);
      if (cudaMemcpy(cond->data(), B.cond, n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) return CCM_ECUDA;
    } else {
      beta->resize(16 * n);
      norm->resize(n);
      ok->resize(n);
      if (cudaMemcpy(beta->data(), B.beta, 16 * n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess ||
          cudaMemcpy(norm->data(), B.norm, n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess ||
          cudaMemcpy(ok->data(), B.ok, n, cudaMemcpyDeviceToHost) != cudaSuccess)
        return CCM_ECUDA;
    }
    return CCM_OK;
  }
};

}  // namespace

std::unique_ptr<FitBatcher> make_device_fitter() { return std::unique_ptr<FitBatcher>(new DeviceFitter()); }

}  // namespace ccm
