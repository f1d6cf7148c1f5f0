// Test shim: runs the library's host-side topology builder without a GPU and
// exposes its arrays to tests/test_topology_host.py (compiled by that test).
#include <cstring>
#include <string>

#include "rve_internal.h"

namespace rvegpu {
static std::string g_shim_error;
void set_error(const std::string& m) { g_shim_error = m; }
int fail(int code, const std::string& m) {
  g_shim_error = m;
  return code;
}
}  // namespace rvegpu

static rvegpu::HostTopology g_topo;

extern "C" {
int shim_build(int64_t n_rve, const int64_t* node_off, const double* X, const int64_t* fiber_off,
               const int32_t* conn, const double* L0, const double* EA, const double* B, const uint8_t* nb,
               int64_t* sizes /* fa, fb, csr, ncsr, free_node_id, pruned */) {
  const int rc = rvegpu::build_topology(n_rve, node_off, X, fiber_off, conn, L0, EA, B, nb, nullptr, g_topo);
  if (rc != 0) return rc;
  sizes[0] = int64_t(g_topo.fa.size());
  sizes[1] = int64_t(g_topo.fb.size());
  sizes[2] = int64_t(g_topo.csr.size());
  sizes[3] = int64_t(g_topo.ncsr.size());
  sizes[4] = int64_t(g_topo.free_node_id.size());
  sizes[5] = g_topo.pruned_fibers;
  return 0;
}
const char* shim_error() { return rvegpu::g_shim_error.c_str(); }
// per RVE: nf na nb node_off fa_off fb_off csr_off csr_len
void shim_meta(int32_t* out) {
  for (size_t r = 0; r < g_topo.meta.size(); ++r) {
    const rvegpu::RveMeta& M = g_topo.meta[r];
    const int32_t v[8] = {M.nf, M.na, M.nb, M.node_off, M.fa_off, M.fb_off, M.csr_off, M.csr_len};
    std::memcpy(out + 8 * r, v, sizeof(v));
  }
}
// active fibers: dx dy dz L0 EA B half_inv_L02 per fiber
void shim_fa(double* out) {
  for (size_t e = 0; e < g_topo.fa.size(); ++e) {
    const rvegpu::FibD& f = g_topo.fa[e];
    const double v[7] = {f.dx, f.dy, f.dz, f.L0, f.EA, f.B, f.half_inv_L02};
    std::memcpy(out + 7 * e, v, sizeof(v));
  }
}
void shim_fij(uint32_t* out) { std::memcpy(out, g_topo.fij.data(), g_topo.fij.size() * sizeof(uint32_t)); }
void shim_csr(uint16_t* out) { std::memcpy(out, g_topo.csr.data(), g_topo.csr.size() * sizeof(uint16_t)); }
void shim_ncsr(uint32_t* out) { std::memcpy(out, g_topo.ncsr.data(), g_topo.ncsr.size() * sizeof(uint32_t)); }
void shim_ncap(float* out) { std::memcpy(out, g_topo.ncap.data(), g_topo.ncap.size() * sizeof(float)); }
void shim_nord(uint16_t* out) { std::memcpy(out, g_topo.nord.data(), g_topo.nord.size() * sizeof(uint16_t)); }
void shim_free_ids(int32_t* out) {
  std::memcpy(out, g_topo.free_node_id.data(), g_topo.free_node_id.size() * sizeof(int32_t));
}
}
