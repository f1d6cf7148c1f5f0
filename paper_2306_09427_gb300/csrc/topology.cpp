// Host-side set-up of an RVE batch: validation, pruning, renumbering and
// the node-centric CSR (Algorithm 2's one-time set-up: connectivity and
// lumped-mass data are built once per RVE on the CPU, Sec. 3.2).
#include <algorithm>
#include <cmath>
#include <deque>
#include <sstream>

#include "rve_internal.h"

namespace rvegpu {

namespace {

std::string at(int64_t r) {
  std::ostringstream o;
  o << "RVE " << r << ": ";
  return o.str();
}

}  // namespace

int build_topology(int64_t n_rve, const int64_t* node_off, const double* X, const int64_t* fiber_off,
                   const int32_t* conn, const double* L0, const double* EA, const double* B,
                   const uint8_t* is_boundary, const double* V0, HostTopology& T) {
  if (n_rve < 0) return fail(RVE_EINVAL, "n_rve must be >= 0");
  if (n_rve > 0 && (!node_off || !fiber_off)) return fail(RVE_EINVAL, "node_off and fiber_off are required");
  if (n_rve > 0 && (node_off[0] != 0 || fiber_off[0] != 0))
    return fail(RVE_EINVAL, "node_off[0] and fiber_off[0] must be 0");
  for (int64_t r = 0; r < n_rve; ++r) {
    if (node_off[r + 1] < node_off[r]) return fail(RVE_EINVAL, at(r) + "node_off decreases");
    if (fiber_off[r + 1] < fiber_off[r]) return fail(RVE_EINVAL, at(r) + "fiber_off decreases");
  }
  const int64_t N = n_rve ? node_off[n_rve] : 0, E = n_rve ? fiber_off[n_rve] : 0;
  if ((N > 0 && (!X || !is_boundary)) || (E > 0 && (!conn || !L0 || !EA || !B)))
    return fail(RVE_EINVAL, "null input array");
  T = HostTopology();
  T.meta.resize(n_rve);
  T.node_off_in.assign(node_off, node_off + n_rve + 1);
  T.X_in.assign(X, X + 3 * N);
  for (int64_t i = 0; i < 3 * N; ++i)
    if (!std::isfinite(X[i])) return fail(RVE_EINVAL, "non-finite node coordinate");

  std::vector<int32_t> deg, adj_off, adj, local;
  std::vector<uint8_t> alive, ok, seen;
  for (int64_t r = 0; r < n_rve; ++r) {
    const int64_t n0 = node_off[r], n = node_off[r + 1] - n0;
    const int64_t e0 = fiber_off[r], ne = fiber_off[r + 1] - e0;
    const uint8_t* nb = is_boundary + n0;
    const double* Xr = X + 3 * n0;
    // validate fibers
    int64_t nbnd = 0;
    for (int64_t i = 0; i < n; ++i) nbnd += nb[i] != 0;
    if (ne > 0 && nbnd == 0) return fail(RVE_EINVAL, at(r) + "has fibers but no boundary node");
    for (int64_t e = 0; e < ne; ++e) {
      const int64_t a = conn[2 * (e0 + e)], b = conn[2 * (e0 + e) + 1];
      if (a < 0 || b < 0 || a >= n || b >= n) return fail(RVE_EINVAL, at(r) + "fiber node id out of range");
      if (a == b) return fail(RVE_EINVAL, at(r) + "fiber joins a node to itself");
      const double l0 = L0[e0 + e], ea = EA[e0 + e], bb = B[e0 + e];
      if (!(l0 > 0.0) || !std::isfinite(l0)) return fail(RVE_EINVAL, at(r) + "rest length must be > 0");
      if (!(ea > 0.0) || !std::isfinite(ea)) return fail(RVE_EINVAL, at(r) + "EA must be > 0");
      if (!(bb >= 0.0) || !std::isfinite(bb)) return fail(RVE_EINVAL, at(r) + "B must be >= 0");
    }
    // adjacency
    deg.assign(n, 0);
    for (int64_t e = 0; e < ne; ++e) {
      deg[conn[2 * (e0 + e)]]++;
      deg[conn[2 * (e0 + e) + 1]]++;
    }
    adj_off.assign(n + 1, 0);
    for (int64_t i = 0; i < n; ++i) adj_off[i + 1] = adj_off[i] + deg[i];
    adj.assign(adj_off[n], 0);
    {
      std::vector<int32_t> fill(adj_off.begin(), adj_off.end() - 1);
      for (int64_t e = 0; e < ne; ++e) {
        adj[fill[conn[2 * (e0 + e)]]++] = int32_t(e);
        adj[fill[conn[2 * (e0 + e) + 1]]++] = int32_t(e);
      }
    }
    // pruning rule 2: strip free nodes of degree <= 1, repeatedly
    alive.assign(ne, 1);
    ok.assign(n, 1);
    std::deque<int32_t> q;
    for (int64_t i = 0; i < n; ++i)
      if (!nb[i] && deg[i] <= 1) q.push_back(int32_t(i));
    while (!q.empty()) {
      const int32_t i = q.front();
      q.pop_front();
      if (!ok[i]) continue;
      ok[i] = 0;
      for (int32_t k = adj_off[i]; k < adj_off[i + 1]; ++k) {
        const int32_t e = adj[k];
        if (!alive[e]) continue;
        alive[e] = 0;
        const int32_t a = conn[2 * (e0 + e)], b = conn[2 * (e0 + e) + 1];
        const int32_t j = (a == i) ? b : a;
        if (ok[j]) {
          --deg[j];
          if (!nb[j] && deg[j] <= 1) q.push_back(j);
        }
      }
    }
    // pruning rule 1: keep free nodes reachable from the boundary
    seen.assign(n, 0);
    for (int64_t i = 0; i < n; ++i)
      if (nb[i]) {
        seen[i] = 1;
        q.push_back(int32_t(i));
      }
    while (!q.empty()) {
      const int32_t i = q.front();
      q.pop_front();
      for (int32_t k = adj_off[i]; k < adj_off[i + 1]; ++k) {
        const int32_t e = adj[k];
        if (!alive[e]) continue;
        const int32_t a = conn[2 * (e0 + e)], b = conn[2 * (e0 + e) + 1];
        const int32_t j = (a == i) ? b : a;
        if (!seen[j] && ok[j]) {
          seen[j] = 1;
          q.push_back(j);
        }
      }
    }
    for (int64_t i = 0; i < n; ++i)
      if (!nb[i] && !seen[i]) ok[i] = 0;
    // renumber free nodes in input order
    local.assign(n, -1);
    int32_t nf = 0;
    for (int64_t i = 0; i < n; ++i)
      if (!nb[i] && ok[i]) {
        local[i] = nf++;
        T.free_node_id.push_back(int32_t(i));
      }
    if (nf > 65534) return fail(RVE_EINVAL, at(r) + "more than 65534 free nodes after pruning");
    RveMeta& M = T.meta[r];
    M.nf = nf;
    M.n_nodes = int32_t(n);
    M.node_off = int32_t(T.ncsr.size());
    M.fa_off = int32_t(T.fa.size());
    M.fb_off = int32_t(T.fb.size());
    M.csr_off = int32_t(T.csr.size());
    double sum_ea = 0.0;
    std::vector<int32_t> act_id(ne, -1);
    int32_t na = 0, nbf = 0;
    for (int64_t e = 0; e < ne; ++e) {
      const int32_t a = conn[2 * (e0 + e)], b = conn[2 * (e0 + e) + 1];
      alive[e] = alive[e] && ok[a] && ok[b];
      if (!alive[e]) {
        T.pruned_fibers++;
        continue;
      }
      sum_ea += EA[e0 + e];
      const FibD f{Xr[3 * b] - Xr[3 * a], Xr[3 * b + 1] - Xr[3 * a + 1], Xr[3 * b + 2] - Xr[3 * a + 2],
                   L0[e0 + e], EA[e0 + e], B[e0 + e]};
      if (nb[a] && nb[b]) {
        T.fb.push_back(f);
        ++nbf;
      } else {
        T.fa.push_back(f);
        const uint32_t ia = nb[a] ? uint32_t(nf) : uint32_t(local[a]);
        const uint32_t ib = nb[b] ? uint32_t(nf) : uint32_t(local[b]);
        T.fij.push_back(ia | (ib << 16));
        act_id[e] = na++;
      }
    }
    if (na > 32767) return fail(RVE_EINVAL, at(r) + "more than 32767 active fibers after pruning");
    M.na = na;
    M.nb = nbf;
    M.sum_EA = sum_ea;
    // node-centric CSR: incident active fibers in increasing fiber order
    for (int64_t i = 0; i < n; ++i) {
      if (local[i] < 0) continue;
      const uint32_t begin = uint32_t(T.csr.size()) - uint32_t(M.csr_off);
      uint32_t cnt = 0;
      double lmin = 1e300;
      std::vector<int32_t> inc;
      for (int32_t k = adj_off[i]; k < adj_off[i + 1]; ++k) {
        const int32_t e = adj[k];
        if (act_id[e] >= 0) inc.push_back(e);
      }
      std::sort(inc.begin(), inc.end());
      for (int32_t e : inc) {
        const bool is_j = conn[2 * (e0 + e) + 1] == int32_t(i);
        T.csr.push_back(uint16_t((uint32_t(act_id[e]) << 1) | (is_j ? 1u : 0u)));
        lmin = std::min(lmin, L0[e0 + e]);
        ++cnt;
      }
      if (cnt > 252) return fail(RVE_EINVAL, at(r) + "a free node has more than 252 fibers");
      // pad the run to a multiple of 4 entries with the zero scratch slot (na)
      while (cnt % 4 != 0) {
        T.csr.push_back(uint16_t(uint32_t(na) << 1));
        ++cnt;
      }
      T.ncsr.push_back((begin << 8) | cnt);
      T.ncap.push_back(float(STEP_CAP * lmin));
    }
    // reference volume
    if (V0) {
      if (!(V0[r] > 0.0) || !std::isfinite(V0[r])) return fail(RVE_EINVAL, at(r) + "V0 must be > 0");
      M.V0 = V0[r];
    } else {
      double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
      for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k) {
          lo[k] = std::min(lo[k], Xr[3 * i + k]);
          hi[k] = std::max(hi[k], Xr[3 * i + k]);
        }
      M.V0 = n ? (hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]) : 1.0;
      if (!(M.V0 > 0.0)) M.V0 = 1.0;
    }
    M.csr_len = int32_t(T.csr.size() - size_t(M.csr_off));
    if (size_t(M.csr_len) >= (1u << 24)) return fail(RVE_EINVAL, at(r) + "CSR too large");
  }
  if (T.ncsr.size() > size_t(INT32_MAX) || T.fa.size() > size_t(INT32_MAX) || T.csr.size() > size_t(INT32_MAX))
    return fail(RVE_EINVAL, "batch too large for 32-bit offsets");
  return RVE_OK;
}

}  // namespace rvegpu
