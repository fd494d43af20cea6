// Host planning: see plan.h.
//
// Ordering.  The pose graphs of the workloads are long, nearly one-dimensional chains
// (sequential and (k, k+2) edges) coupled by a few inter-agent or loop edges.  A
// minimum-degree ordering eliminates such chains from their ends and yields an
// elimination tree as deep as the chain, which serialises the factorisation.  Nested
// dissection by breadth-first level structures (a middle BFS level from a
// pseudo-peripheral node is a vertex separator; both sides are ordered recursively,
// the separator last) keeps the tree depth logarithmic at a small cost in fill, which
// matters on a GPU where every tree level is a dependent FP64 step.
#include "plan.h"

#include <algorithm>
#include <cmath>
#include <numeric>
#include <set>

namespace como3r {
namespace {

constexpr int kLeaf = 4;

struct Dissector {
  const std::vector<std::vector<int>>& adj;
  std::vector<int> tag;
  std::vector<int> dist;
  int next_tag = 0;
  std::vector<int> order;

  explicit Dissector(const std::vector<std::vector<int>>& a) : adj(a), tag(a.size(), -1), dist(a.size(), -1) {}

  // BFS levels of the nodes tagged t reachable from `start`.
  std::vector<std::vector<int>> levels_from(int start, int t) {
    std::vector<std::vector<int>> lv;
    std::vector<int> touched{start};
    dist[start] = 0;
    lv.push_back({start});
    while (true) {
      std::vector<int> nxt;
      for (int u : lv.back())
        for (int w : adj[u])
          if (tag[w] == t && dist[w] < 0) {
            dist[w] = (int)lv.size();
            nxt.push_back(w);
            touched.push_back(w);
          }
      if (nxt.empty()) break;
      std::sort(nxt.begin(), nxt.end());
      lv.push_back(std::move(nxt));
    }
    for (int v : touched) dist[v] = -1;
    return lv;
  }

  void run(std::vector<int> nodes) {
    if ((int)nodes.size() <= kLeaf) {
      std::sort(nodes.begin(), nodes.end());
      order.insert(order.end(), nodes.begin(), nodes.end());
      return;
    }
    const int t = next_tag++;
    for (int v : nodes) tag[v] = t;
    std::sort(nodes.begin(), nodes.end());
    auto lv = levels_from(nodes[0], t);
    size_t reached = 0;
    for (auto& l : lv) reached += l.size();
    if (reached < nodes.size()) {  // several components: order each separately
      std::vector<std::vector<int>> comps;
      std::vector<char> seen(adj.size(), 0);
      for (int v : nodes) {
        if (seen[v]) continue;
        auto cl = levels_from(v, t);
        std::vector<int> comp;
        for (auto& l : cl)
          for (int u : l) {
            seen[u] = 1;
            comp.push_back(u);
          }
        comps.push_back(std::move(comp));
      }
      for (auto& c : comps) run(std::move(c));
      return;
    }
    for (int rep = 0; rep < 4; ++rep) {  // pseudo-peripheral start node
      int far = -1, best_deg = 1 << 30;
      for (int u : lv.back()) {
        int deg = 0;
        for (int w : adj[u]) deg += (tag[w] == t);
        if (deg < best_deg || (deg == best_deg && u < far)) {
          best_deg = deg;
          far = u;
        }
      }
      auto l2 = levels_from(far, t);
      if (l2.size() <= lv.size()) break;
      lv = std::move(l2);
    }
    const int h = (int)lv.size();
    if (h < 3) {
      order.insert(order.end(), nodes.begin(), nodes.end());
      return;
    }
    const int lo = std::max(1, h / 3), hi = std::min(h - 2, (2 * h) / 3);
    int m = lo;
    for (int k = lo; k <= hi; ++k) {
      const bool smaller = lv[k].size() < lv[m].size();
      const bool tie_closer = lv[k].size() == lv[m].size() && std::abs(k - h / 2) < std::abs(m - h / 2);
      if (smaller || tie_closer) m = k;
    }
    std::vector<int> A, B;
    for (int k = 0; k < m; ++k) A.insert(A.end(), lv[k].begin(), lv[k].end());
    for (int k = m + 1; k < h; ++k) B.insert(B.end(), lv[k].begin(), lv[k].end());
    std::vector<int> S = lv[m];
    run(std::move(A));
    run(std::move(B));
    std::sort(S.begin(), S.end());
    order.insert(order.end(), S.begin(), S.end());
  }
};

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

}  // namespace

int build_plan(const como3r_graph_desc* d, HostPlan& p) {
  auto fail = [&](const std::string& msg) {
    p.error = msg;
    return COMO3R_ERR_INVALID_ARG;
  };
  if (!d) return fail("desc is NULL");
  if (d->num_graphs < 1) return fail("num_graphs must be >= 1");
  if (!d->kf_offset || !d->height || !d->width || !d->edge_offset || !d->edge_i || !d->edge_j)
    return fail("kf_offset, height, width, edge_offset, edge_i and edge_j must be non-NULL");
  if (!(finite_pos(d->sigma_ray) && finite_pos(d->sigma_dist) && finite_pos(d->huber_k) && finite_pos(d->eps0)))
    return fail("sigma_ray, sigma_dist, huber_k and eps0 must be finite and > 0");
  if (!(std::isfinite(d->lambda) && d->lambda >= 0.0)) return fail("lambda must be finite and >= 0");
  if (d->max_attempts < 1 || d->max_attempts > 16) return fail("max_attempts must be in 1..16");
  if (d->mode != COMO3R_PLAIN_FP64 && d->mode != COMO3R_MIXED) return fail("unknown mode");
  if (d->dtype < COMO3R_F16 || d->dtype > COMO3R_F64) return fail("unknown dtype");
  const int G = d->num_graphs;
  p.G = G;
  p.mode = d->mode;
  p.dtype = d->dtype;
  p.kf_offset.assign(d->kf_offset, d->kf_offset + G + 1);
  p.edge_offset.assign(d->edge_offset, d->edge_offset + G + 1);
  if (p.kf_offset[0] != 0 || p.edge_offset[0] != 0) return fail("kf_offset[0] and edge_offset[0] must be 0");
  for (int g = 0; g < G; ++g) {
    if (p.kf_offset[g + 1] <= p.kf_offset[g]) return fail("every graph needs >= 1 keyframe (kf_offset increasing)");
    if (p.edge_offset[g + 1] < p.edge_offset[g]) return fail("edge_offset must be non-decreasing");
    if (d->height[g] <= 0 || d->width[g] <= 0) return fail("height and width must be > 0");
    if ((int64_t)d->height[g] * d->width[g] >= (int64_t(1) << 30)) return fail("pointmap larger than 2^30 pixels");
  }
  const int N = p.kf_offset[G], E = p.edge_offset[G];
  p.N = N;
  p.E = E;
  if (!d->points_conf) return fail("points_conf is NULL");
  if (E > 0 && !d->match_idx) return fail("match_idx is NULL");
  if (E >= (1 << 29)) return fail("too many edges");
  p.npix.resize(N);
  p.pix_off.assign(N + 1, 0);
  for (int g = 0; g < G; ++g)
    for (int k = p.kf_offset[g]; k < p.kf_offset[g + 1]; ++k) p.npix[k] = d->height[g] * d->width[g];
  for (int k = 0; k < N; ++k) p.pix_off[k + 1] = p.pix_off[k] + p.npix[k];
  p.total_px = p.pix_off[N];
  // anchors
  p.anchor.resize(G);
  for (int g = 0; g < G; ++g) {
    int a = p.kf_offset[g];
    if (d->anchor) {
      a = d->anchor[g];
      if (a < p.kf_offset[g] || a >= p.kf_offset[g + 1]) return fail("anchor outside its graph");
    } else if (d->agent_of) {
      for (int k = p.kf_offset[g]; k < p.kf_offset[g + 1]; ++k)
        if (d->agent_of[k] < d->agent_of[a]) a = k;
    }
    p.anchor[g] = a;
  }
  p.frozen.assign(N, 0);
  for (int g = 0; g < G; ++g) p.frozen[p.anchor[g]] = 1;
  // edges
  p.es.resize(E);
  int64_t off = 0;
  for (int g = 0; g < G; ++g)
    for (int e = p.edge_offset[g]; e < p.edge_offset[g + 1]; ++e) {
      const int i = d->edge_i[e], j = d->edge_j[e];
      if (i < p.kf_offset[g] || i >= p.kf_offset[g + 1] || j < p.kf_offset[g] || j >= p.kf_offset[g + 1])
        return fail("edge endpoint outside its graph (edge " + std::to_string(e) + ")");
      if (i == j) return fail("edge with i == j (edge " + std::to_string(e) + ")");
      EdgeStatic s{};
      s.pix_i = p.pix_off[i];
      s.pix_j = p.pix_off[j];
      s.idx_off = off;
      s.i = i;
      s.j = j;
      s.npix_i = p.npix[i];
      s.npix_j = p.npix[j];
      p.es[e] = s;
      off += p.npix[i];
    }
  p.total_idx = off;

  // ---- per graph: ordering, symbolic factorisation, levels
  p.col_begin.assign(1, 0);
  p.col_slot.assign(1, 0);
  p.tri_off.assign(1, 0);
  p.rs_off.assign(1, 0);
  p.lvl_begin.assign(1, 0);
  p.lvl_off.assign(1, 0);
  std::vector<std::vector<int32_t>> slot_lists;  // contributions per slot
  std::vector<std::vector<int32_t>> kf_lists(N);
  for (int g = 0; g < G; ++g) {
    const int k0 = p.kf_offset[g], nk = p.kf_offset[g + 1] - k0, a = p.anchor[g] - k0;
    // local node ids (anchor removed): node u <-> keyframe k0 + kf_of[u]
    std::vector<int> node_of(nk, -1), kf_of;
    for (int l = 0; l < nk; ++l)
      if (l != a) {
        node_of[l] = (int)kf_of.size();
        kf_of.push_back(l);
      }
    const int n = (int)kf_of.size();
    std::vector<std::vector<int>> adj(n);
    for (int e = p.edge_offset[g]; e < p.edge_offset[g + 1]; ++e) {
      const int u = node_of[d->edge_i[e] - k0], v = node_of[d->edge_j[e] - k0];
      if (u < 0 || v < 0) continue;
      adj[u].push_back(v);
      adj[v].push_back(u);
    }
    for (auto& l : adj) {
      std::sort(l.begin(), l.end());
      l.erase(std::unique(l.begin(), l.end()), l.end());
    }
    Dissector nd(adj);
    std::vector<int> all(n);
    std::iota(all.begin(), all.end(), 0);
    nd.run(all);
    std::vector<int> pos(n);
    for (int q = 0; q < n; ++q) pos[nd.order[q]] = q;
    // symbolic elimination on positions
    std::vector<std::set<int>> nb(n);
    for (int u = 0; u < n; ++u)
      for (int v : adj[u]) nb[pos[u]].insert(pos[v]);
    std::vector<std::vector<int>> rows(n);
    for (int k = 0; k < n; ++k) {
      rows[k].assign(nb[k].begin(), nb[k].end());  // all > k: earlier columns were removed
      for (int r : rows[k]) {
        nb[r].erase(k);
        for (int r2 : rows[k])
          if (r2 != r) nb[r].insert(r2);
      }
      nb[k].clear();
    }
    // levels
    std::vector<int> level(n, 0);
    int nlev = n ? 1 : 0;
    for (int k = 0; k < n; ++k)
      if (!rows[k].empty()) {
        level[rows[k][0]] = std::max(level[rows[k][0]], level[k] + 1);
        nlev = std::max(nlev, level[rows[k][0]] + 1);
      }
    p.max_levels = std::max(p.max_levels, nlev);
    // columns and slots (global numbering)
    const int cbase = p.col_begin.back();
    std::vector<int> slot_base(n);
    for (int k = 0; k < n; ++k) {
      p.col_kf.push_back(k0 + kf_of[nd.order[k]]);
      slot_base[k] = p.col_slot.back();
      p.slot_row.push_back(cbase + k);  // diagonal
      for (int r : rows[k]) p.slot_row.push_back(cbase + r);
      p.col_slot.push_back(slot_base[k] + 1 + (int)rows[k].size());
    }
    auto slot_of = [&](int r, int c) {  // block (r, c), r >= c, of this graph
      if (r == c) return slot_base[c];
      const auto it = std::lower_bound(rows[c].begin(), rows[c].end(), r);
      return slot_base[c] + 1 + (int)(it - rows[c].begin());
    };
    for (int k = 0; k < n; ++k) {
      const int kc = p.col_kf[cbase + k];
      p.slot_kf_r.push_back(kc);
      p.slot_kf_c.push_back(kc);
      for (int r : rows[k]) {
        p.slot_kf_r.push_back(p.col_kf[cbase + r]);
        p.slot_kf_c.push_back(kc);
      }
    }
    // row structure and left-looking update triplets
    std::vector<std::vector<int>> rowstruct(n);
    for (int j = 0; j < n; ++j)
      for (int r : rows[j]) rowstruct[r].push_back(j);
    for (int k = 0; k < n; ++k) {
      std::vector<std::pair<int, int4>> ts;
      for (int j : rowstruct[k]) {
        p.rs.push_back(make_int2(slot_of(k, j), cbase + j));
        for (int r : rows[j])
          if (r >= k) ts.push_back({j, make_int4(slot_of(r, j), slot_of(k, j), slot_of(r, k), 0)});
      }
      std::stable_sort(ts.begin(), ts.end(), [](const auto& x, const auto& y) {
        return x.second.z != y.second.z ? x.second.z < y.second.z : x.first < y.first;
      });
      for (auto& t : ts) p.tri.push_back(t.second);
      p.tri_off.push_back((int)p.tri.size());
      p.rs_off.push_back((int)p.rs.size());
    }
    // level schedule
    std::vector<int> byl(n);
    std::iota(byl.begin(), byl.end(), 0);
    std::stable_sort(byl.begin(), byl.end(), [&](int x, int y) { return level[x] < level[y]; });
    for (int q = 0; q < n; ++q) {
      p.sched.push_back(cbase + byl[q]);
      if (q + 1 == n || level[byl[q + 1]] != level[byl[q]]) p.lvl_off.push_back((int)p.sched.size());
    }
    p.lvl_begin.push_back((int)p.lvl_off.size() - 1);
    p.col_begin.push_back(cbase + n);
    // assembly contributions
    slot_lists.resize(p.col_slot.back());
    for (int e = p.edge_offset[g]; e < p.edge_offset[g + 1]; ++e) {
      const int i = d->edge_i[e], j = d->edge_j[e];
      const int ui = node_of[i - k0], uj = node_of[j - k0];
      if (ui >= 0) {
        slot_lists[slot_of(pos[ui], pos[ui])].push_back(2 * e);
        kf_lists[i].push_back(2 * e + 1);
      }
      if (uj >= 0) {
        slot_lists[slot_of(pos[uj], pos[uj])].push_back(2 * e);
        kf_lists[j].push_back(2 * e);
      }
      if (ui >= 0 && uj >= 0) {
        const int r = std::max(pos[ui], pos[uj]), c = std::min(pos[ui], pos[uj]);
        slot_lists[slot_of(r, c)].push_back(2 * e + 1);
      }
    }
    const size_t nslot = (size_t)(p.col_slot.back() - p.col_slot[cbase]);
    p.max_graph_smem = std::max(p.max_graph_smem, sizeof(double) * (nslot * 49 + (size_t)n * 14));
  }
  p.slot_contrib_off.assign(1, 0);
  for (auto& l : slot_lists) {
    if (l.empty()) ++p.fill_blocks;
    p.slot_contrib.insert(p.slot_contrib.end(), l.begin(), l.end());
    p.slot_contrib_off.push_back((int)p.slot_contrib.size());
  }
  p.kf_contrib_off.assign(1, 0);
  for (auto& l : kf_lists) {
    p.kf_contrib.insert(p.kf_contrib.end(), l.begin(), l.end());
    p.kf_contrib_off.push_back((int)p.kf_contrib.size());
  }
  return COMO3R_OK;
}

void build_items(const HostPlan& p, int chunk, std::vector<Item>& items, std::vector<int32_t>& item_off) {
  items.clear();
  item_off.assign(1, 0);
  for (int e = 0; e < p.E; ++e) {
    const int P = p.es[e].npix_i;
    for (int b = 0; b < P; b += chunk) items.push_back(Item{e, b, std::min(b + chunk, P), 0});
    item_off.push_back((int)items.size());
  }
}

void plan_stats(const HostPlan& p, int64_t* s) {
  for (int k = 0; k < COMO3R_STAT_COUNT; ++k) s[k] = 0;
  s[COMO3R_STAT_GRAPHS] = p.G;
  s[COMO3R_STAT_KEYFRAMES] = p.N;
  s[COMO3R_STAT_EDGES] = p.E;
  s[COMO3R_STAT_COLUMNS] = p.col_begin.empty() ? 0 : p.col_begin.back();
  s[COMO3R_STAT_BLOCKS] = p.col_slot.empty() ? 0 : p.col_slot.back();
  s[COMO3R_STAT_FILL] = p.fill_blocks;
  s[COMO3R_STAT_UPDATES] = (int64_t)p.tri.size();
  s[COMO3R_STAT_LEVELS] = p.max_levels;
}

}  // namespace como3r
