// The setup's work on the GPU.  The batched fits (FitBatcher of host.h): the level's cut-cell
// moments, volumes and boundary-piece moments go to the device once per call, the (row,
// candidate) pairs as index lists, and k_plg_fit / k_plg_cond return the coefficients, the
// weighted norms and the condition numbers.  The centre classification (CentreClassifier):
// one thread per cell tests its centre against every curve.  Blocking; device memory is
// released before returning.
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

namespace dev {

// a curve for the centre test (the inside tests of Curve::inside)
struct CentreCurve {
  int kind, orient, npoly;
  double p[8];
  const double* poly;   // polygon vertices or the spline's polyline (x0, y0, x1, y1, ...)
};

__device__ bool centre_inside(const CentreCurve& c, double x, double y) {
  if (c.kind == CCM_POLYGON || c.kind == CCM_SPLINE) {
    // even-odd rule: a ray towards +x crosses the closed polyline an odd number of times
    bool in = false;
    for (int k = 0; k < c.npoly; ++k) {
      const double xa = c.poly[2 * k], ya = c.poly[2 * k + 1];
      const int k1 = k + 1 == c.npoly ? 0 : k + 1;
      const double xb = c.poly[2 * k1], yb = c.poly[2 * k1 + 1];
      if (ya == yb) continue;
      if ((ya > y) != (yb > y) && x < xa + (y - ya) * (xb - xa) / (yb - ya)) in = !in;
    }
    return in;
  }
  const double dx = x - c.p[0], dy = y - c.p[1];
  if (c.kind == CCM_CIRCLE) return dx * dx + dy * dy < c.p[2] * c.p[2];
  if (c.kind == CCM_ELLIPSE) {
    const double cs = cos(c.p[4]), sn = sin(c.p[4]);
    const double X = (dx * cs + dy * sn) / c.p[2], Y = (-dx * sn + dy * cs) / c.p[3];
    return X * X + Y * Y < 1.0;
  }
  return hypot(dx, dy) < c.p[2] + c.p[3] * cos(c.p[4] * atan2(dy, dx));
}

// one thread per cell: ST_PURE when the centre is inside every curve with orient +1 and
// outside every curve with orient -1, else ST_EMPTY
__global__ void k_classify_centres(int nx, int ny, double x0, double y0, double h, int nc,
                                   const CentreCurve* __restrict__ curves, int8_t* __restrict__ status) {
  const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long)nx * ny) return;
  const int i = (int)(q % nx), j = (int)(q / nx);
  const double x = x0 + (i + 0.5) * h, y = y0 + (j + 0.5) * h;
  bool in = true;
  for (int k = 0; k < nc && in; ++k)
    if ((curves[k].orient > 0) != centre_inside(curves[k], x, y)) in = false;
  status[q] = in ? (int8_t)ST_PURE : (int8_t)ST_EMPTY;
}

}  // namespace dev

namespace {

class DeviceClassifier final : public CentreClassifier {
 public:
  int classify(const CutLevel& cg, std::vector<int8_t>& status) override {
    const long N = (long)cg.nx * cg.ny;
    status.resize(N);
    DevBufs D;
    std::vector<dev::CentreCurve> cv(cg.curves.size());
    for (size_t k = 0; k < cg.curves.size(); ++k) {
      const Curve& c = cg.curves[k];
      dev::CentreCurve& d = cv[k];
      d.kind = c.kind;
      d.orient = c.orient;
      std::memcpy(d.p, c.p, sizeof(d.p));
      const std::vector<double>* P = c.kind == CCM_POLYGON ? &c.V : c.kind == CCM_SPLINE ? &c.poly : nullptr;
      d.npoly = P ? (int)(P->size() / 2) : 0;
      d.poly = P ? D.put(*P) : nullptr;
    }
    const dev::CentreCurve* dcv = D.put(cv);
    int8_t* ds = D.get<int8_t>(N);
    if (D.err != cudaSuccess) return D.err == cudaErrorMemoryAllocation ? CCM_ENOMEM : CCM_ECUDA;
    dev::k_classify_centres<<<(unsigned)((N + 255) / 256), 256>>>(cg.nx, cg.ny, cg.x0, cg.y0, cg.h,
                                                                  (int)cv.size(), dcv, ds);
    if (cudaGetLastError() != cudaSuccess) return CCM_ECUDA;
    if (cudaMemcpy(status.data(), ds, N, cudaMemcpyDeviceToHost) != cudaSuccess) return CCM_ECUDA;
    return CCM_OK;
  }
};

}  // namespace

std::unique_ptr<CentreClassifier> make_device_classifier() {
  return std::unique_ptr<CentreClassifier>(new DeviceClassifier());
}

}  // namespace ccm
