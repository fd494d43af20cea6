// Host planning: see plan.h.
//
// Ordering.  The pose graphs of the workloads are long, nearly one-dimensional chains
// (sequential and (k, k+2) edges) coupled by a few inter-agent or loop edges.  A
// minimum-degree ordering eliminates such chains from their ends and yields an
// elimination tree as deep as the chain, which serialises the factorisation.  Nested
// dissection by breadth-first level structures (a middle BFS level from a
// pseudo-peripheral node is a vertex separator; both sides are ordered recursively,
// the separator last) keeps the tree depth logarithmic at a small cost in fill, which
// matters on a GPU where every tree level is a dependent FP64 step.  For graphs with
// more cross-links a minimum-degree order can be both shallower in fill and not much
// deeper; each graph takes whichever of the two a simple cost model rates cheaper
// (levels x per-level latency + block updates x per-update FP64 time).
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

// Exact minimum-degree elimination order on the (small) block graph; ties -> lowest id.
std::vector<int> min_degree_order(const std::vector<std::vector<int>>& adj) {
  const int n = (int)adj.size();
  std::vector<std::set<int>> G(n);
  for (int u = 0; u < n; ++u) G[u].insert(adj[u].begin(), adj[u].end());
  std::vector<char> done(n, 0);
  std::vector<int> order;
  order.reserve(n);
  for (int step = 0; step < n; ++step) {
    int v = -1;
    size_t best = SIZE_MAX;
    for (int u = 0; u < n; ++u)
      if (!done[u] && G[u].size() < best) {
        best = G[u].size();
        v = u;
      }
    done[v] = 1;
    order.push_back(v);
    std::vector<int> nb(G[v].begin(), G[v].end());
    for (int a : nb) {
      G[a].erase(v);
      for (int b : nb)
        if (b != a) G[a].insert(b);
    }
    G[v].clear();
  }
  return order;
}

struct Symbolic {
  std::vector<int> pos;                 // node -> elimination position
  std::vector<std::vector<int>> rows;   // per position: sorted rows > position
  std::vector<int> level;               // per position: elimination-tree level
  int nlev = 0;
  int64_t updates = 0;
};

Symbolic symbolic(const std::vector<std::vector<int>>& adj, const std::vector<int>& order) {
  const int n = (int)adj.size();
  Symbolic S;
  S.pos.assign(n, 0);
  for (int q = 0; q < n; ++q) S.pos[order[q]] = q;
  std::vector<std::set<int>> nb(n);
  for (int u = 0; u < n; ++u)
    for (int v : adj[u]) nb[S.pos[u]].insert(S.pos[v]);
  S.rows.assign(n, {});
  for (int k = 0; k < n; ++k) {
    S.rows[k].assign(nb[k].begin(), nb[k].end());  // all > k: earlier columns were removed
    for (int r : S.rows[k]) {
      nb[r].erase(k);
      for (int r2 : S.rows[k])
        if (r2 != r) nb[r].insert(r2);
    }
    nb[k].clear();
    const int64_t c = (int64_t)S.rows[k].size();
    S.updates += c * (c + 1) / 2;
  }
  S.level.assign(n, 0);
  S.nlev = n ? 1 : 0;
  for (int k = 0; k < n; ++k)
    if (!S.rows[k].empty()) {
      S.level[S.rows[k][0]] = std::max(S.level[S.rows[k][0]], S.level[k] + 1);
      S.nlev = std::max(S.nlev, S.level[S.rows[k][0]] + 1);
    }
  return S;
}

// Rough cost (microseconds) of one factorisation + solve on one SM: every level pays
// the dependent-latency chain of a 7x7 factorisation and the substitutions, every
// block update ~14 warp FP64 instructions at one per 20 cycles.
double order_cost(const Symbolic& S) { return 3.0 * S.nlev + 0.15 * (double)S.updates; }

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

}  // namespace

int build_plan(const como3r_graph_desc* d, HostPlan& p, const std::vector<int8_t>* force_order) {
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
  p.width.assign(d->width, d->width + G);
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
  // Fixed keyframes: the anchor of each graph, plus the lowest keyframe of every other
  // connected component (a component not joined to the anchor's keeps a deterministic
  // reference of its own, so no gauge direction is left to the eps regulariser).
  p.frozen.assign(N, 0);
  {
    std::vector<int> parent(N);
    std::iota(parent.begin(), parent.end(), 0);
    auto find = [&](int a) {
      while (parent[a] != a) a = parent[a] = parent[parent[a]];
      return a;
    };
    for (int e = 0; e < p.edge_offset[G]; ++e) {
      const int a = find(d->edge_i[e]), b = find(d->edge_j[e]);
      if (a != b) parent[std::max(a, b)] = std::min(a, b);
    }
    for (int g = 0; g < G; ++g) {
      std::vector<char> has_fixed(N, 0);
      has_fixed[find(p.anchor[g])] = 1;
      p.frozen[p.anchor[g]] = 1;
      for (int k = p.kf_offset[g]; k < p.kf_offset[g + 1]; ++k) {
        const int r = find(k);
        if (!has_fixed[r]) {
          has_fixed[r] = 1;
          p.frozen[k] = 1;
        }
      }
    }
  }

  // ---- per graph: ordering, symbolic factorisation, levels
  p.col_begin.assign(1, 0);
  p.slot_begin.assign(1, 0);
  int lvl_base = 0;
  std::vector<std::vector<int32_t>> slot_lists;  // contributions per slot
  std::vector<std::vector<int32_t>> kf_lists(N);
  for (int g = 0; g < G; ++g) {
    const int k0 = p.kf_offset[g], nk = p.kf_offset[g + 1] - k0;
    // local node ids (fixed keyframes removed): node u <-> keyframe k0 + kf_of[u]
    std::vector<int> node_of(nk, -1), kf_of;
    for (int l = 0; l < nk; ++l)
      if (!p.frozen[k0 + l]) {
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
    Symbolic S_nd = symbolic(adj, nd.order);
    const std::vector<int> md_order = min_degree_order(adj);
    Symbolic S_md = symbolic(adj, md_order);
    const int forced = force_order && g < (int)force_order->size() ? (*force_order)[g] : -1;
    const bool use_md = forced >= 0 ? forced == 0 : order_cost(S_md) <= order_cost(S_nd);
    p.nlev_md.push_back(S_md.nlev);
    p.nlev_nd.push_back(S_nd.nlev);
    p.upd_md.push_back(S_md.updates);
    p.upd_nd.push_back(S_nd.updates);
    const std::vector<int>& order = use_md ? md_order : nd.order;
    Symbolic& S = use_md ? S_md : S_nd;
    p.order_kind.push_back(use_md ? 0 : 1);
    const std::vector<int>& pos = S.pos;
    const std::vector<std::vector<int>>& rows = S.rows;
    const std::vector<int>& level = S.level;
    p.max_levels = std::max(p.max_levels, S.nlev);
    // columns and slots: local numbering inside the graph, global = base + local
    const int cbase = p.col_begin.back(), sbase = p.slot_begin.back();
    std::vector<int> slot_base(n);  // local slot of each column's diagonal block
    int nslot = 0;
    for (int k = 0; k < n; ++k) {
      p.col_kf.push_back(k0 + kf_of[order[k]]);
      slot_base[k] = nslot;
      p.col_slot.push_back(sbase + nslot);
      p.lcol_slot.push_back(nslot);
      p.lslot_row.push_back(k);  // diagonal
      for (int r : rows[k]) p.lslot_row.push_back(r);
      nslot += 1 + (int)rows[k].size();
    }
    p.lcol_slot.push_back(nslot);
    auto slot_of = [&](int r, int c) {  // local slot of block (r, c), r >= c
      if (r == c) return slot_base[c];
      const auto it = std::lower_bound(rows[c].begin(), rows[c].end(), r);
      return slot_base[c] + 1 + (int)(it - rows[c].begin());
    };
    // blocks of L by block row (the left-looking forward substitution with a kept factor):
    // row r lists (slot of L_rj, j) for j < r in ascending j
    {
      std::vector<int> cnt(n + 1, 0);
      for (int k = 0; k < n; ++k)
        for (int r : rows[k]) ++cnt[r + 1];
      for (int r = 0; r < n; ++r) cnt[r + 1] += cnt[r];
      const size_t e0 = p.lrow_ent.size();
      p.lrow_ent.resize(e0 + (size_t)cnt[n]);
      std::vector<int> fill(cnt.begin(), cnt.end() - 1);
      for (int k = 0; k < n; ++k)
        for (int r : rows[k]) p.lrow_ent[e0 + (size_t)fill[r]++] = make_int2(slot_of(r, k), k);
      p.lrow_off.insert(p.lrow_off.end(), cnt.begin(), cnt.end());
    }
    for (int k = 0; k < n; ++k) {
      const int kc = p.col_kf[cbase + k];
      p.slot_kf_r.push_back(kc);
      p.slot_kf_c.push_back(kc);
      for (int r : rows[k]) {
        p.slot_kf_r.push_back(p.col_kf[cbase + r]);
        p.slot_kf_c.push_back(kc);
      }
    }
    // right-looking update triplets: after the columns of a level are factored, their
    // contributions L_rj L_kj^T go to every ancestor block (r, k); the triplets of one
    // source level are grouped by destination block (local indices)
    std::vector<std::vector<std::pair<int, int4>>> trip_of_level(S.nlev);
    for (int j = 0; j < n; ++j)
      for (size_t a = 0; a < rows[j].size(); ++a)
        for (size_t b = 0; b <= a; ++b) {
          const int r = rows[j][a], k = rows[j][b];
          trip_of_level[level[j]].push_back({j, make_int4(slot_of(r, j), slot_of(k, j), slot_of(r, k), j)});
        }
    const int tri0 = (int)p.ltri.size();
    std::vector<int> diag_col(nslot, -1);
    for (int k = 0; k < n; ++k) diag_col[slot_base[k]] = k;
    std::vector<std::vector<int4>> tasks_of_level(S.nlev);
    for (int lv = 0; lv < S.nlev; ++lv) {
      auto& ts = trip_of_level[lv];
      std::stable_sort(ts.begin(), ts.end(), [](const auto& x, const auto& y) {
        return x.second.z != y.second.z ? x.second.z < y.second.z : x.first < y.first;
      });
      size_t q = 0;
      while (q < ts.size()) {
        size_t e = q;
        while (e < ts.size() && ts[e].second.z == ts[q].second.z) ++e;
        const int dst = ts[q].second.z;
        const int t0 = (int)p.ltri.size() - tri0;
        for (size_t x = q; x < e; ++x) p.ltri.push_back(ts[x].second);
        // a diagonal destination also receives the forward right-hand side of its column
        tasks_of_level[lv].push_back(make_int4(dst, t0, (int)p.ltri.size() - tri0, diag_col[dst]));
        q = e;
      }
    }
    // level schedule: columns, off-diagonal solve tasks, update tasks (longest first)
    std::vector<int> byl(n);
    std::iota(byl.begin(), byl.end(), 0);
    std::stable_sort(byl.begin(), byl.end(), [&](int x, int y) { return level[x] < level[y]; });
    // the level of the column that owns each local slot
    std::vector<int> level_of_slot(nslot);
    for (int k = 0; k < n; ++k)
      for (int sl = slot_base[k]; sl < slot_base[k] + 1 + (int)rows[k].size(); ++sl) level_of_slot[sl] = level[k];
    const int u0 = (int)p.lutask.size(), t0 = (int)p.lttask.size();
    int q = 0;
    for (int lv = 0; lv < S.nlev; ++lv) {
      const int sched0 = q, tt0 = (int)p.lttask.size() - t0;
      int qe = q, max_nb = 0;
      for (; qe < n && level[byl[qe]] == lv; ++qe) max_nb = std::max(max_nb, (int)rows[byl[qe]].size());
      // a narrow level (at most kPanelCols columns, each with at most kPanelBlocks
      // off-diagonal blocks, or one column with at most kPanel4Blocks) is factored as whole
      // column panels: its off-diagonal rows ride along in the diagonal elimination, so it
      // gets no off-diagonal solve tasks
      const bool panel = (qe - q <= kPanelCols && max_nb <= kPanelBlocks) || (qe - q == 1 && max_nb <= kPanel4Blocks);
      for (; q < qe; ++q) {
        const int k = byl[q];
        p.lsched.push_back(k);
        if (!panel)
          for (size_t b = 0; b < rows[k].size(); ++b) p.lttask.push_back(make_int2(slot_base[k] + 1 + (int)b, k));
      }
      // updates into the next level's columns ("near", needed by its factorisation) first,
      // then the rest ("far", which the kernel overlaps with the next level's diagonal
      // factorisations); longest first within each kind
      auto& tl = tasks_of_level[lv];
      std::stable_sort(tl.begin(), tl.end(), [&](const int4& x, const int4& y) {
        const bool nx = level_of_slot[x.x] == lv + 1, ny = level_of_slot[y.x] == lv + 1;
        if (nx != ny) return nx;
        return (x.z - x.y) > (y.z - y.y);
      });
      const int un0 = (int)p.lutask.size() - u0;
      int n_near = 0;
      for (const int4& t : tl) n_near += level_of_slot[t.x] == lv + 1;
      p.lutask.insert(p.lutask.end(), tl.begin(), tl.end());
      p.llvl.insert(p.llvl.end(), {sched0, un0, un0 + n_near, tt0});
    }
    {
      const int nu_all = (int)p.lutask.size() - u0;
      p.llvl.insert(p.llvl.end(), {q, nu_all, nu_all, (int)p.lttask.size() - t0});
    }
    const int ntri = (int)p.ltri.size() - tri0, nu = (int)p.lutask.size() - u0, nt = (int)p.lttask.size() - t0;
    p.meta.insert(p.meta.end(), {cbase, n, sbase, nslot, tri0, ntri, u0, nu, t0, nt, lvl_base, S.nlev});
    lvl_base += S.nlev + 1;
    p.col_begin.push_back(cbase + n);
    p.slot_begin.push_back(sbase + nslot);
    p.max_graph_smem = std::max(p.max_graph_smem, solver_smem_bytes(nslot, n, ntri, nu, nt, S.nlev));
    // assembly contributions (global slots)
    slot_lists.resize(p.slot_begin.back());
    for (int e = p.edge_offset[g]; e < p.edge_offset[g + 1]; ++e) {
      const int i = d->edge_i[e], j = d->edge_j[e];
      const int ui = node_of[i - k0], uj = node_of[j - k0];
      if (ui >= 0) {
        slot_lists[sbase + slot_of(pos[ui], pos[ui])].push_back(2 * e);
        kf_lists[i].push_back(2 * e + 1);
      }
      if (uj >= 0) {
        slot_lists[sbase + slot_of(pos[uj], pos[uj])].push_back(2 * e);
        kf_lists[j].push_back(2 * e);
      }
      if (ui >= 0 && uj >= 0) {
        const int r = std::max(pos[ui], pos[uj]), c = std::min(pos[ui], pos[uj]);
        slot_lists[sbase + slot_of(r, c)].push_back(2 * e + 1);
      }
    }
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
  s[COMO3R_STAT_BLOCKS] = p.slot_begin.empty() ? 0 : p.slot_begin.back();
  s[COMO3R_STAT_FILL] = p.fill_blocks;
  s[COMO3R_STAT_UPDATES] = (int64_t)p.ltri.size();
  s[COMO3R_STAT_LEVELS] = p.max_levels;
  int64_t nd = 0;
  for (int8_t k : p.order_kind) nd += k;
  s[COMO3R_STAT_ND_GRAPHS] = nd;
  // FP64 operations of one factorisation and solve (an FMA counts 2): per column the 7x7
  // Cholesky (140) with its right-hand side (49), L_cc^{-1} (114) and the back-substitution
  // product with it (56); per off-diagonal block the triangular solve (343) and its
  // back-substitution product (98); per update triplet a 7x7x7 product (686), and 98 more
  // when the destination is diagonal (the right-hand side rides along).
  const int64_t cols = s[COMO3R_STAT_COLUMNS], offdiag = s[COMO3R_STAT_BLOCKS] - cols;
  int64_t rhs_tri = 0;
  for (const int4& t : p.lutask)
    if (t.w >= 0) rhs_tri += t.z - t.y;
  s[COMO3R_STAT_SOLVE_FLOPS] = cols * (140 + 49 + 114 + 56) + offdiag * (343 + 98) +
                               (int64_t)p.ltri.size() * 686 + rhs_tri * 98;
  s[COMO3R_STAT_SOLVE_GROUPS] = 0;  // the device's choice (como3r_graph_stats)
}


void build_cluster_plan(const HostPlan& p, int C, HostClusterPlan& cp) {
  cp = HostClusterPlan{};
  cp.C = C;
  cp.slot_home.assign(p.slot_begin.back(), 0);
  cp.col_home.assign(p.col_begin.back(), 0);
  for (int g = 0; g < p.G; ++g) {
    const int* m = p.meta.data() + kMetaCount * g;
    const int cbase = m[kMetaColBase], ncol = m[kMetaNCol], sbase = m[kMetaSlotBase], nslot = m[kMetaNSlot];
    const int ubase = m[kMetaUBase], tbase = m[kMetaTBase], nlev = m[kMetaNLvl], tribase = m[kMetaTriBase];
    const int* lvl = p.llvl.data() + 4 * m[kMetaLvlBase];
    const int* colslot = p.lcol_slot.data() + cbase + g;
    const int* sched = p.lsched.data() + cbase;
    // owners: per level, each column (largest first: 1 + its off-diagonal blocks, the
    // factorisation and off-diagonal solve work) to the CTA with the least work of the level
    // so far, lowest rank on ties -- so the narrow top of the elimination tree (one column
    // per level) stays on rank 0 and its near updates read local shared memory, and the
    // wide bottom levels end together; the far updates are spread below
    std::vector<int> owner(ncol, 0), clocal(ncol, 0), slocal(nslot, 0), shome(nslot, 0);
    std::vector<std::vector<int>> own_cols(C), own_slots(C);
    for (int l = 0; l < nlev; ++l) {
      std::vector<int> cols(sched + lvl[4 * l], sched + lvl[4 * (l + 1)]);
      auto cost = [&](int c) { return colslot[c + 1] - colslot[c]; };
      std::stable_sort(cols.begin(), cols.end(), [&](int a, int b) { return cost(a) > cost(b); });
      std::vector<int> load(C, 0);
      for (int c : cols) {
        int best = 0;
        for (int r = 1; r < C; ++r)
          if (load[r] < load[best]) best = r;
        owner[c] = best;
        load[best] += cost(c);
      }
    }
    for (int q = 0; q < ncol; ++q) {  // level order
      const int c = sched[q], r = owner[c];
      clocal[c] = (int)own_cols[r].size();
      own_cols[r].push_back(c);
      for (int sl = colslot[c]; sl < colslot[c + 1]; ++sl) {
        shome[sl] = r;
        slocal[sl] = (int)own_slots[r].size();
        own_slots[r].push_back(sl);
      }
    }
    for (int c = 0; c < ncol; ++c) cp.col_home[cbase + c] = (owner[c] << 24) | clocal[c];
    // the top run of levels whose columns are all rank 0's
    int top_local = nlev;
    while (top_local > 0) {
      bool all0 = true;
      for (int q = lvl[4 * (top_local - 1)]; q < lvl[4 * top_local]; ++q) all0 = all0 && owner[sched[q]] == 0;
      if (!all0) break;
      --top_local;
    }
    int ncol_max = 0;
    for (int r = 0; r < C; ++r) ncol_max = std::max(ncol_max, (int)own_cols[r].size());
    for (int sl = 0; sl < nslot; ++sl) cp.slot_home[sbase + sl] = (shome[sl] << 24) | slocal[sl];
    // Executors of the far update tasks of level l (they run during level l + 1's diagonal
    // factorisations, writing their destinations through the cluster window when remote):
    // each task (work = its triplets) goes to the CTA with the least estimated work so far,
    // where a CTA that factors columns of level l + 1 starts from that factorisation's time
    // (kFarBusyBase triplets' worth per round of up to kClusterPanelCols columns: on this GPU
    // an SM's FP64 pipe is narrow, and updates run beside a critical factorisation delay it)
    // and an idle CTA from zero; ties go to the highest rank (rank 0 owns the critical top
    // of the tree).  So the idle CTAs take the far work first, and it spreads over every CTA
    // only where it would outlast the factorisations (a wide level under a level with one
    // idle CTA).
    constexpr long long kFarBusyBase = 24;
    std::vector<int> far_exec(std::max(lvl[4 * nlev + 1], 0), -1);
    for (int l = 0; l < nlev; ++l) {
      std::vector<long long> load(C, 0);
      if (l + 1 < nlev) {
        std::vector<int> nown(C, 0);
        for (int q = lvl[4 * (l + 1)]; q < lvl[4 * (l + 2)]; ++q) ++nown[owner[sched[q]]];
        for (int r = 0; r < C; ++r)
          if (nown[r]) load[r] = kFarBusyBase * ((nown[r] + kClusterPanelCols - 1) / kClusterPanelCols);
      }
      for (int u = lvl[4 * l + 2]; u < lvl[4 * (l + 1) + 1]; ++u) {
        const int4 t = p.lutask[ubase + u];
        int best = C - 1;
        for (int r = C - 2; r >= 0; --r)
          if (load[r] < load[best]) best = r;
        far_exec[u] = best;
        load[best] += std::max(1, t.z - t.y);
      }
    }
    for (int r = 0; r < C; ++r) {
      const int s0 = (int)cp.csched.size(), u0 = (int)cp.cutask.size(), t0 = (int)cp.cttask.size();
      const int l0 = (int)cp.clvl.size(), o0 = (int)cp.own_slot.size();
      for (int l = 0; l < nlev; ++l) {
        const int sc = (int)cp.csched.size() - s0, un = (int)cp.cutask.size() - u0;
        for (int q = lvl[4 * l]; q < lvl[4 * (l + 1)]; ++q)
          if (owner[sched[q]] == r) cp.csched.push_back(sched[q]);
        int nn = 0;
        for (int u = lvl[4 * l + 1]; u < lvl[4 * l + 2]; ++u) {
          const int4 t = p.lutask[ubase + u];
          if (shome[t.x] == r) {
            cp.cutask.push_back(t);
            ++nn;
          }
        }
        for (int u = lvl[4 * l + 2]; u < lvl[4 * (l + 1) + 1]; ++u)
          if (far_exec[u] == r) cp.cutask.push_back(p.lutask[ubase + u]);
        const int tt = (int)cp.cttask.size() - t0;
        // this CTA factors its columns of the level as whole panels (no off-diagonal solve
        // tasks) when it owns at most kClusterPanelCols of them, each with at most
        // kPanelBlocks off-diagonal blocks (one warp per column), or a single one with at
        // most kPanel4Blocks (four warps)
        int n_own = 0, max_nb = 0;
        for (int q = lvl[4 * l]; q < lvl[4 * (l + 1)]; ++q)
          if (owner[sched[q]] == r) {
            ++n_own;
            max_nb = std::max(max_nb, colslot[sched[q] + 1] - colslot[sched[q]] - 1);
          }
        const bool panel_cta = (n_own <= kClusterPanelCols && max_nb <= kPanelBlocks) ||
                               (n_own == 1 && max_nb <= kPanel4Blocks);
        if (!panel_cta)
          for (int x = lvl[4 * l + 3]; x < lvl[4 * (l + 1) + 3]; ++x) {
            const int2 t = p.lttask[tbase + x];
            if (shome[t.x] == r) cp.cttask.push_back(t);
          }
        cp.clvl.insert(cp.clvl.end(), {sc, un, un + nn, tt});
      }
      cp.clvl.insert(cp.clvl.end(), {(int)cp.csched.size() - s0, (int)cp.cutask.size() - u0,
                                     (int)cp.cutask.size() - u0, (int)cp.cttask.size() - t0});
      // this CTA's triplets, in the order of its tasks, which are re-pointed at them
      const int r0 = (int)cp.ctri.size();
      for (size_t u = u0; u < cp.cutask.size(); ++u) {
        int4& t = cp.cutask[u];
        const int b = (int)cp.ctri.size() - r0;
        cp.ctri.insert(cp.ctri.end(), p.ltri.begin() + tribase + t.y, p.ltri.begin() + tribase + t.z);
        t.z = b + (t.z - t.y);
        t.y = b;
      }
      const int nrt = (int)cp.ctri.size() - r0;
      for (int sl : own_slots[r]) cp.own_slot.push_back(sl);
      const int nsl = (int)own_slots[r].size(), ncl = (int)own_cols[r].size();
      cp.cmeta.insert(cp.cmeta.end(), {s0, (int)cp.csched.size() - s0, u0, (int)cp.cutask.size() - u0, t0,
                                       (int)cp.cttask.size() - t0, l0, nsl, ncl, o0, ncol_max, top_local, r0, nrt});
      cp.max_cta_smem = std::max(cp.max_cta_smem,
                                 cluster_smem_bytes(nsl, ncl, ncol_max, nrt, (int)cp.cutask.size() - u0,
                                                    (int)cp.cttask.size() - t0, nlev, nslot, ncol));
    }
  }
}

}  // namespace como3r

namespace como3r {

// Estimated solve times (microseconds), fitted to one-CTA solves of the 64-graph batch on
// this GPU (per-graph completion stamps): one CTA with the factor in global memory pays
// ~40 us per graph (staging, the first attempt's set-up), ~6.3 us per elimination level (a
// 7x7 factorisation chain with L2 round trips) and ~0.26 us per block update (14 FP64 warp
// instructions on one SM's four sub-partitions, with their loads); a cluster of kGroupCTAs
// pays ~10 us per level (cluster barriers) and spreads the updates over its SMs.
void build_group_plan(const HostPlan& p, int sms, int force_big, GroupPlan& gp) {
  gp = GroupPlan();
  const int G = p.G;
  if (G < 2 || sms < kGroupCTAs) return;
  auto one = [&](int g) {
    const bool md = 3.0 * p.nlev_md[g] + 0.15 * (double)p.upd_md[g] <= 3.0 * p.nlev_nd[g] + 0.15 * (double)p.upd_nd[g];
    return 40.0 + (md ? 6.3 * p.nlev_md[g] + 0.26 * (double)p.upd_md[g] : 6.3 * p.nlev_nd[g] + 0.26 * (double)p.upd_nd[g]);
  };
  auto group = [&](int g, int* order) {
    const double md = 10.0 * p.nlev_md[g] + 0.26 / kGroupCTAs * (double)p.upd_md[g];
    const double nd = 10.0 * p.nlev_nd[g] + 0.26 / kGroupCTAs * (double)p.upd_nd[g];
    if (order) *order = md <= nd ? 0 : 1;
    return md <= nd ? md : nd;
  };
  std::vector<int> idx(G);
  std::iota(idx.begin(), idx.end(), 0);
  std::vector<double> e1(G);
  for (int g = 0; g < G; ++g) e1[g] = one(g);
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return e1[a] > e1[b]; });
  gp.single_us = e1[idx[0]];
  // the remaining graphs, largest first, each onto the least-loaded of m CTAs
  auto pack = [&](int k, int m, std::vector<std::vector<int>>* bins) {
    std::vector<double> load(m, 0.0);
    if (bins) bins->assign(m, {});
    for (int q = k; q < G; ++q) {
      const int b = (int)(std::min_element(load.begin(), load.end()) - load.begin());
      load[b] += e1[idx[q]];
      if (bins) (*bins)[b].push_back(idx[q]);
    }
    return m ? *std::max_element(load.begin(), load.end()) : 0.0;
  };
  int best_k = -1, best_m = 0;
  double best = 0.8 * gp.single_us;  // a group solve must gain at least a fifth
  const int kmax = std::min(G, sms / kGroupCTAs);
  for (int k = 1; k <= kmax; ++k) {
    if (force_big >= 0 && k != force_big) continue;
    // the CTAs left for the other graphs, whole clusters (none when every graph is clustered)
    const int m = k < G ? ((sms - kGroupCTAs * k) / kGroupCTAs) * kGroupCTAs : 0;
    if (k < G && m == 0) continue;
    double mk = pack(k, m, nullptr);
    for (int q = 0; q < k; ++q) mk = std::max(mk, group(idx[q], nullptr));
    if (force_big >= 0 || mk < best) {
      best = mk;
      best_k = k;
      best_m = m;
    }
  }
  if (best_k < 1) return;
  gp.big = best_k;
  gp.makespan_us = best;
  gp.order.assign(G, -1);
  for (int q = 0; q < best_k; ++q) {
    int o = 0;
    group(idx[q], &o);
    gp.order[idx[q]] = (int8_t)o;
    const int off = (int)gp.glist.size();
    gp.glist.push_back(idx[q]);
    for (int r = 0; r < kGroupCTAs; ++r) gp.gtask.push_back(make_int4(off, 1, r, kGroupCTAs));
  }
  std::vector<std::vector<int>> bins;
  pack(best_k, best_m, &bins);
  for (const auto& b : bins) {
    gp.gtask.push_back(make_int4((int)gp.glist.size(), (int)b.size(), 0, 1));
    for (int g : b) gp.glist.push_back(g);
  }
  gp.ctas = (int)gp.gtask.size();
}

}  // namespace como3r
