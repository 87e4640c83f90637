// Host-only view of the setup (include/ccm.h, ccm_host_*): builds the hierarchy without
// touching a device so that the discrete choices can be inspected on any machine.
#include <cstring>
#include <memory>

#include "hierarchy.h"

struct ccm_host_setup {
  ccm::Hierarchy H;
};

extern "C" {

int ccm_default_params(ccm_params* p);

int ccm_host_build(const ccm_problem* prob, const ccm_params* params, ccm_host_setup** out) {
  if (!prob || !out) return CCM_EINVAL;
  *out = nullptr;
  if (int rc = ccm::check_problem(*prob)) return rc;
  ccm_params par;
  ccm_default_params(&par);
  if (params) par = *params;
  std::unique_ptr<ccm_host_setup> s(new ccm_host_setup());
  std::string err;
  int rc = ccm::build_hierarchy(*prob, par, s->H, err);
  if (rc) return rc;
  *out = s.release();
  return CCM_OK;
}

int ccm_host_level_sizes(const ccm_host_setup* s, int level, int* nx, int* ny, int64_t* n2, int64_t* nseg) {
  if (!s || level < 0 || level >= (int)s->H.levels.size()) return CCM_EINVAL;
  const ccm::HostLevel& L = s->H.levels[level];
  if (nx) *nx = L.nx;
  if (ny) *ny = L.ny;
  if (n2) *n2 = L.n2;
  if (nseg) *nseg = (int64_t)s->H.cut[level].segs.size();
  return CCM_OK;
}

int ccm_host_rows(const ccm_host_setup* s, int level, int32_t* cell, int32_t* cols, double* beta, double* nb,
                  int32_t* seg) {
  if (!s) return CCM_EINVAL;
  return ccm::hierarchy_rows(s->H, level, cell, cols, beta, nb, seg);
}

int ccm_host_cell_map(const ccm_host_setup* s, int level, int8_t* status, int32_t* owner, int8_t* regular,
                      double* vol, double* mom) {
  if (!s || level < 0 || level >= (int)s->H.levels.size()) return CCM_EINVAL;
  const ccm::CutLevel& c = s->H.cut[level];
  const ccm::HostLevel& L = s->H.levels[level];
  long n = (long)c.nx * c.ny;
  if (status) std::memcpy(status, c.status.data(), n);
  if (owner) std::memcpy(owner, c.owner.data(), n * sizeof(int32_t));
  if (vol) std::memcpy(vol, c.vol.data(), n * sizeof(double));
  if (regular)
    for (int j = 0; j < c.ny; ++j)
      for (int i = 0; i < c.nx; ++i) regular[(long)j * c.nx + i] = L.cls[L.pad(i, j)] == 1 ? 1 : 0;
  if (mom)
    for (long q = 0; q < n; ++q) {
      const ccm::Mom& m = c.status[q] == ccm::ST_EMPTY ? ccm::Mom{} : c.moments((int)q);
      for (int k = 0; k < ccm::NMOM; ++k) mom[q * ccm::NMOM + k] = m[k];
    }
  return CCM_OK;
}

void ccm_host_free(ccm_host_setup* s) { delete s; }

}  // extern "C"
