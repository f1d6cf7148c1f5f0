// Host-side set-up of an RVE batch: validation, pruning, renumbering and
// the node-centric CSR (Algorithm 2's one-time set-up: connectivity and
// lumped-mass data are built once per RVE on the CPU, Sec. 3.2).
#include <algorithm>
#include <cmath>
#include <deque>
#include <sstream>
#include <thread>

#include "rve_internal.h"

namespace rvegpu {

namespace {

std::string at(int64_t r) {
  std::ostringstream o;
  o << "RVE " << r << ": ";
  return o.str();
}

// Shared-memory bank layout.  The kernels gather 16-byte rows (H[i], H[j]
// per fiber; SCR[e] per CSR entry); a warp's 16-byte load is served in four
// phases of 8 lanes, and two lanes of a phase conflict when they read
// different rows whose indices agree mod 8 (the same four banks).  Both the
// order of the active fibers and the order of the entries inside a node's
// run of 4 are free, so they are chosen here, once per RVE, to keep rows
// read in one phase in different bank groups.

// Phase bookkeeping: distinct row indices seen per residue class mod 8.
struct PhaseClasses {
  int32_t v[8][8];
  int n[8];
  void clear() {
    for (int k = 0; k < 8; ++k) n[k] = 0;
  }
  // rows of class x % 8 already in the phase that differ from x
  int cost(int32_t x) const {
    const int k = x & 7;
    for (int t = 0; t < n[k]; ++t)
      if (v[k][t] == x) return 0;
    return n[k];
  }
  void add(int32_t x) {
    const int k = x & 7;
    for (int t = 0; t < n[k]; ++t)
      if (v[k][t] == x) return;
    if (n[k] < 8) v[k][n[k]++] = x;
  }
};

// Order of the active fibers: consecutive groups of 8 fibers (one load phase
// of the fiber loop) are filled greedily; each slot takes, among the next
// ORDER_WINDOW unplaced fibers, the first that adds no conflict to the H[i]
// and H[j] loads of its group, else the one adding the fewest.
constexpr int ORDER_WINDOW = 1024;

std::vector<int32_t> fiber_order(const std::vector<uint32_t>& ij) {
  const int32_t na = int32_t(ij.size());
  std::vector<int32_t> next(size_t(na) + 1), prev(size_t(na) + 1), out;
  out.reserve(size_t(na));
  // doubly linked list of unplaced fibers; node na is the head sentinel
  for (int32_t e = 0; e < na; ++e) {
    next[e] = e + 1;
    prev[e] = e - 1;
  }
  next[na] = na ? 0 : na;
  if (na) prev[0] = na;
  if (na) next[na - 1] = na;
  PhaseClasses ci, cj;
  while (int32_t(out.size()) < na) {
    ci.clear();
    cj.clear();
    for (int slot = 0; slot < 8 && int32_t(out.size()) < na; ++slot) {
      int32_t best = -1, best_cost = 1 << 30, seen = 0;
      for (int32_t c = next[na]; c != na && seen < ORDER_WINDOW; c = next[c], ++seen) {
        const int32_t k = ci.cost(int32_t(ij[c] & 0xffffu)) + cj.cost(int32_t(ij[c] >> 16));
        if (k < best_cost) {
          best = c;
          best_cost = k;
          if (k == 0) break;
        }
      }
      out.push_back(best);
      ci.add(int32_t(ij[best] & 0xffffu));
      cj.add(int32_t(ij[best] >> 16));
      next[prev[best]] = next[best];
      prev[next[best]] = prev[best];
    }
  }
  return out;
}

// Order inside the CSR runs: for each group of 8 consecutive free nodes (one
// load phase of the gather) and each run of 4 entries, the nodes with the
// most real entries (not the zero slot na) first pick the permutation of their 4 entries adding the
// fewest conflicts at the 4 load positions.
void order_runs(std::vector<std::vector<uint16_t>>& runs, uint32_t na) {
  static const uint8_t perm[24][4] = {
      {0, 1, 2, 3}, {0, 1, 3, 2}, {0, 2, 1, 3}, {0, 2, 3, 1}, {0, 3, 1, 2}, {0, 3, 2, 1},
      {1, 0, 2, 3}, {1, 0, 3, 2}, {1, 2, 0, 3}, {1, 2, 3, 0}, {1, 3, 0, 2}, {1, 3, 2, 0},
      {2, 0, 1, 3}, {2, 0, 3, 1}, {2, 1, 0, 3}, {2, 1, 3, 0}, {2, 3, 0, 1}, {2, 3, 1, 0},
      {3, 0, 1, 2}, {3, 0, 2, 1}, {3, 1, 0, 2}, {3, 1, 2, 0}, {3, 2, 0, 1}, {3, 2, 1, 0}};
  const size_t nf = runs.size();
  for (size_t g0 = 0; g0 < nf; g0 += 8) {
    const size_t g1 = std::min(nf, g0 + 8);
    size_t rounds = 0;
    for (size_t a = g0; a < g1; ++a) rounds = std::max(rounds, runs[a].size() / 4);
    for (size_t rd = 0; rd < rounds; ++rd) {
      PhaseClasses pos[4];
      for (auto& p : pos) p.clear();
      std::vector<std::pair<int, size_t>> nodes;  // (-real entries, node)
      for (size_t a = g0; a < g1; ++a) {
        if (runs[a].size() <= 4 * rd) continue;
        int real = 0;
        for (int t = 0; t < 4; ++t) real += (uint32_t(runs[a][4 * rd + t]) >> 1) != na ? 1 : 0;
        nodes.push_back({-real, a});
      }
      std::stable_sort(nodes.begin(), nodes.end());
      for (const auto& na_ : nodes) {
        uint16_t* e = runs[na_.second].data() + 4 * rd;
        int best = 0, best_cost = 1 << 30;
        for (int p = 0; p < 24; ++p) {
          int k = 0;
          for (int t = 0; t < 4; ++t) k += pos[t].cost(int32_t(e[perm[p][t]] >> 1));
          if (k < best_cost) {
            best = p;
            best_cost = k;
            if (k == 0) break;
          }
        }
        const uint16_t o[4] = {e[0], e[1], e[2], e[3]};
        for (int t = 0; t < 4; ++t) {
          e[t] = o[perm[best][t]];
          pos[t].add(int32_t(e[t] >> 1));
        }
      }
    }
  }
}

// Applies both orders to RVE r: permutes its active fibers, renames the CSR
// entries to the new fiber indices, sorts each run and orders its entries.
void order_rve(HostTopology& T, int64_t r) {
  const RveMeta& M = T.meta[size_t(r)];
  const size_t f0 = size_t(M.fa_off), na = size_t(M.na);
  const std::vector<uint32_t> ij(T.fij.begin() + f0, T.fij.begin() + f0 + na);
  const std::vector<FibD> fd(T.fa.begin() + f0, T.fa.begin() + f0 + na);
  const std::vector<int32_t> ord = fiber_order(ij);
  std::vector<uint16_t> pos(na + 1);
  for (size_t k = 0; k < na; ++k) {
    T.fij[f0 + k] = ij[size_t(ord[k])];
    T.fa[f0 + k] = fd[size_t(ord[k])];
    pos[size_t(ord[k])] = uint16_t(k);
  }
  pos[na] = uint16_t(na);
  std::vector<std::vector<uint16_t>> runs(static_cast<size_t>(M.nf));
  uint16_t* csr = T.csr.data() + M.csr_off;
  for (int32_t a = 0; a < M.nf; ++a) {
    const uint32_t w = T.ncsr[size_t(M.node_off + a)];
    auto& run = runs[size_t(a)];
    run.assign(csr + (w >> 8), csr + (w >> 8) + (w & 0xffu));
    for (auto& x : run) x = uint16_t((uint32_t(pos[x >> 1]) << 1) | (x & 1u));
    std::sort(run.begin(), run.end());  // the zero slot na sorts last
  }
  order_runs(runs, uint32_t(na));
  for (int32_t a = 0; a < M.nf; ++a) {
    const uint32_t w = T.ncsr[size_t(M.node_off + a)];
    std::copy(runs[size_t(a)].begin(), runs[size_t(a)].end(), csr + (w >> 8));
  }
  // free nodes by decreasing degree (ties by index): the node-centric kernel
  // deals them to threads in this order, so the nodes a warp owns at one
  // time have (nearly) the same number of fibers
  std::vector<std::pair<int, int32_t>> by_deg(static_cast<size_t>(M.nf));
  for (int32_t a = 0; a < M.nf; ++a) {
    int real = 0;
    for (uint16_t x : runs[size_t(a)]) real += (uint32_t(x) >> 1) != na ? 1 : 0;
    by_deg[size_t(a)] = {-real, a};
  }
  std::sort(by_deg.begin(), by_deg.end());
  for (int32_t k = 0; k < M.nf; ++k) T.nord[size_t(M.node_off + k)] = uint16_t(by_deg[size_t(k)].second);
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
                   L0[e0 + e], EA[e0 + e], B[e0 + e],
                   0.5 / (L0[e0 + e] * L0[e0 + e])};
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
    // node-centric CSR: the incident active fibers of every free node (in
    // local order), runs padded to a multiple of 4 with the zero scratch slot na
    std::vector<std::vector<uint16_t>> runs(static_cast<size_t>(nf));
    for (int64_t i = 0; i < n; ++i) {
      if (local[i] < 0) continue;
      std::vector<uint16_t>& run = runs[size_t(local[i])];
      double lmin = 1e300;
      for (int32_t k = adj_off[i]; k < adj_off[i + 1]; ++k) {
        const int32_t e = adj[k];
        if (act_id[e] < 0) continue;
        const bool is_j = conn[2 * (e0 + e) + 1] == int32_t(i);
        run.push_back(uint16_t((uint32_t(act_id[e]) << 1) | (is_j ? 1u : 0u)));
        lmin = std::min(lmin, L0[e0 + e]);
      }
      if (run.size() > 252) return fail(RVE_EINVAL, at(r) + "a free node has more than 252 fibers");
      std::sort(run.begin(), run.end());
      while (run.size() % 4 != 0) run.push_back(uint16_t(uint32_t(na) << 1));
      T.ncap.push_back(float(STEP_CAP * lmin));
    }
    for (const auto& run : runs) {
      const uint32_t begin = uint32_t(T.csr.size()) - uint32_t(M.csr_off);
      T.csr.insert(T.csr.end(), run.begin(), run.end());
      T.ncsr.push_back((begin << 8) | uint32_t(run.size()));
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
  // bank-aware orders; every RVE owns disjoint segments, so RVEs run on
  // separate host threads
  const int64_t n_thr = std::max<int64_t>(1, std::min<int64_t>(std::thread::hardware_concurrency(), n_rve / 16));
  T.nord.assign(T.ncsr.size(), 0);
  std::vector<std::thread> pool;
  for (int64_t t = 0; t < n_thr; ++t)
    pool.emplace_back([&T, t, n_thr, n_rve] {
      for (int64_t r = t; r < n_rve; r += n_thr) order_rve(T, r);
    });
  for (auto& th : pool) th.join();
  return RVE_OK;
}

}  // namespace rvegpu
