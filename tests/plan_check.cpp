// Host-side checks of the multi-SM solver's plan (build_cluster_plan), compiled and run by
// tests/test_plan_host.py.  For synthetic pose-graph topologies and cluster sizes 2..16:
//   * every update task of the graph's plan is run exactly once per level: a near task by
//     the CTA that owns its destination, a far task by one executor;
//   * a CTA's tasks index its own triplet list, and the triplets they reach there are the
//     triplets of the same task in the graph's list, in the same order;
//   * far tasks are assigned greedily by estimated work: a CTA's last far task of a level
//     went to it while its estimated work was the least of all CTAs;
//   * the shared memory reported covers every CTA's blocks, scratch, triplets and lists;
//   * the symbolic factorisation, levels and update triplets (see check_symbolic);
//   * the CTA-group plan of a batch (see check_groups).
// Prints "OK <checks>" on success, "FAIL <reason>" otherwise.
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "plan.h"

using namespace como3r;

namespace {

int g_checks = 0;
#define CHECK(cond, ...)                 \
  do {                                   \
    ++g_checks;                          \
    if (!(cond)) {                       \
      std::printf("FAIL ");              \
      std::printf(__VA_ARGS__);          \
      std::printf("\n");                 \
      std::exit(1);                      \
    }                                    \
  } while (0)

struct Topo {
  std::string name;
  std::vector<int32_t> kf_offset, height, width, agent_of, edge_offset, edge_i, edge_j, anchor;
};

// Graphs of `agents` chains of n keyframes each: consecutive edges, skip edges every
// second keyframe, loop closures every `loop` keyframes and `inter` edges between agents.
void add_graph(Topo& t, int agents, int n, int loop, int inter, unsigned seed) {
  const int base = t.kf_offset.back();
  for (int a = 0; a < agents; ++a)
    for (int k = 0; k < n; ++k) t.agent_of.push_back(a);
  auto kf = [&](int a, int k) { return base + a * n + k; };
  for (int a = 0; a < agents; ++a) {
    for (int k = 0; k + 1 < n; ++k) t.edge_i.push_back(kf(a, k)), t.edge_j.push_back(kf(a, k + 1));
    for (int k = 0; k + 2 < n; k += 2) t.edge_i.push_back(kf(a, k)), t.edge_j.push_back(kf(a, k + 2));
    if (loop > 0)
      for (int k = loop; k < n; k += loop) t.edge_i.push_back(kf(a, k - loop)), t.edge_j.push_back(kf(a, k));
  }
  unsigned s = seed;
  auto rnd = [&](int m) { s = s * 1664525u + 1013904223u; return (int)((s >> 8) % (unsigned)m); };
  for (int q = 0; q < inter && agents > 1; ++q) {
    const int a = rnd(agents), b = (a + 1 + rnd(agents - 1)) % agents;
    t.edge_i.push_back(kf(a, rnd(n)));
    t.edge_j.push_back(kf(b, rnd(n)));
  }
  t.kf_offset.push_back(base + agents * n);
  t.height.push_back(48);
  t.width.push_back(64);
  t.edge_offset.push_back((int32_t)t.edge_i.size());
  t.anchor.push_back(base);
}

void check_topology(const Topo& t) {
  const int G = (int)t.height.size();
  float dummy[4] = {0, 0, 0, 0};
  int32_t midx[1] = {-1};
  como3r_graph_desc d{};
  d.num_graphs = G;
  d.kf_offset = t.kf_offset.data();
  d.height = t.height.data();
  d.width = t.width.data();
  d.agent_of = t.agent_of.data();
  d.points_conf = dummy;
  d.dtype = COMO3R_F32;
  d.edge_offset = t.edge_offset.data();
  d.edge_i = t.edge_i.data();
  d.edge_j = t.edge_j.data();
  d.match_idx = midx;
  d.anchor = t.anchor.data();
  d.sigma_ray = 0.003;
  d.sigma_dist = 10;
  d.huber_k = 1.345;
  d.eps0 = 1e-6;
  d.max_attempts = 6;
  d.mode = COMO3R_MIXED;
  HostPlan p;
  CHECK(build_plan(&d, p) == COMO3R_OK, "%s: build_plan: %s", t.name.c_str(), p.error.c_str());
  for (int C : {2, 4, 8, 16}) {
    HostClusterPlan cp;
    build_cluster_plan(p, C, cp);
    for (int g = 0; g < G; ++g) {
      const int* m = p.meta.data() + kMetaCount * g;
      const int nlev = m[kMetaNLvl], ubase = m[kMetaUBase], tribase = m[kMetaTriBase], sbase = m[kMetaSlotBase];
      const int cbase = m[kMetaColBase];
      const int* lvl = p.llvl.data() + 4 * m[kMetaLvlBase];
      const int* colslot = p.lcol_slot.data() + cbase + g;
      // per level: global tasks by destination slot
      for (int l = 0; l < nlev; ++l) {
        std::map<int, int> seen;  // destination -> times run
        std::vector<long long> load(C, 0), last_w(C, 0);
        std::vector<int> nown_next(C, 0);
        for (int r = 0; r < C; ++r) {
          const int32_t* cm = cp.cmeta.data() + kCMetaCount * (g * C + r);
          const int32_t* L = cp.clvl.data() + cm[kCLvl];
          if (l + 1 < nlev) nown_next[r] = L[4 * (l + 1) + 4] - L[4 * (l + 1)];
          const int4* ut = cp.cutask.data() + cm[kCU];
          const int4* ct = cp.ctri.data() + cm[kCTri];
          // near tasks of level l: [L[4l+1], L[4l+2]); far: [L[4l+2], L[4(l+1)+1])
          for (int u = L[4 * l + 1]; u < L[4 * (l + 1) + 1]; ++u) {
            const int4 tk = ut[u];
            const bool near = u < L[4 * l + 2];
            CHECK(tk.y >= 0 && tk.y <= tk.z && tk.z <= cm[kCNTri], "%s C=%d rank %d: task %d triplets [%d,%d) "
                  "outside its list of %d", t.name.c_str(), C, r, u, tk.y, tk.z, cm[kCNTri]);
            // the same destination among the graph's tasks of this level
            int found = -1;
            for (int v = lvl[4 * l + 1]; v < lvl[4 * (l + 1) + 1]; ++v)
              if (p.lutask[ubase + v].x == tk.x) found = v;
            CHECK(found >= 0, "%s C=%d rank %d level %d: destination %d not a task of the level", t.name.c_str(), C,
                  r, l, tk.x);
            const int4 gt = p.lutask[ubase + found];
            CHECK(near == (found < lvl[4 * l + 2]), "%s C=%d: near/far kind changed for destination %d",
                  t.name.c_str(), C, tk.x);
            CHECK(gt.w == tk.w && gt.z - gt.y == tk.z - tk.y, "%s C=%d: task of destination %d changed",
                  t.name.c_str(), C, tk.x);
            for (int q = 0; q < tk.z - tk.y; ++q) {
              const int4 a = ct[tk.y + q], b = p.ltri[tribase + gt.y + q];
              CHECK(a.x == b.x && a.y == b.y && a.z == b.z && a.w == b.w, "%s C=%d rank %d: triplet %d of "
                    "destination %d differs from the graph's", t.name.c_str(), C, r, q, tk.x);
            }
            if (near) {
              const int h = cp.slot_home[sbase + tk.x];
              CHECK((h >> 24) == r, "%s C=%d: near task of destination %d run by rank %d, owned by rank %d",
                    t.name.c_str(), C, tk.x, r, h >> 24);
            } else {
              const long long w = std::max(1, tk.z - tk.y);
              load[r] += w;
              last_w[r] = w;
            }
            ++seen[tk.x];
          }
        }
        for (int v = lvl[4 * l + 1]; v < lvl[4 * (l + 1) + 1]; ++v) {
          const int dst = p.lutask[ubase + v].x;
          CHECK(seen[dst] == 1, "%s C=%d level %d: destination %d run %d times", t.name.c_str(), C, l, dst,
                seen[dst]);
        }
        // greedy far assignment: the last far task of each executor went to it while its
        // estimated work (a factorising CTA's base + far work so far) was the least
        std::vector<long long> total(C);
        for (int r = 0; r < C; ++r) {
          const long long base = nown_next[r] ? 24LL * ((nown_next[r] + kClusterPanelCols - 1) / kClusterPanelCols) : 0;
          total[r] = base + load[r];
        }
        for (int r = 0; r < C; ++r) {
          if (last_w[r] == 0) continue;
          for (int q = 0; q < C; ++q)
            CHECK(total[r] - last_w[r] <= total[q], "%s C=%d level %d: rank %d's last far task taken at work %lld "
                  "while rank %d ends at %lld", t.name.c_str(), C, l, r, total[r] - last_w[r], q, total[q]);
        }
      }
      // shared memory of every CTA within the reported maximum; triplets partitioned
      long long tri_sum = 0, tri_tasks = 0;
      for (int v = 0; v < m[kMetaNU]; ++v) tri_tasks += p.lutask[ubase + v].z - p.lutask[ubase + v].y;
      for (int r = 0; r < C; ++r) {
        const int32_t* cm = cp.cmeta.data() + kCMetaCount * (g * C + r);
        tri_sum += cm[kCNTri];
        const size_t b = cluster_smem_bytes(cm[kCNSlot], cm[kCNCol], cm[kCNColMax], cm[kCNTri], cm[kCNU], cm[kCNT],
                                            nlev, m[kMetaNSlot], m[kMetaNCol]);
        CHECK(b <= cp.max_cta_smem, "%s C=%d rank %d: %zu bytes above the reported %zu", t.name.c_str(), C, r, b,
              cp.max_cta_smem);
      }
      CHECK(tri_sum == tri_tasks, "%s C=%d: %lld triplets staged for %lld in tasks", t.name.c_str(), C, tri_sum,
            tri_tasks);
      (void)colslot;
    }
  }
}

// The symbolic block factorisation and its level schedule, from first principles: in the
// plan's column order, eliminating a column connects all its later neighbours (fill), so
// column c's off-diagonal block rows must be exactly its later neighbours at that point;
// a column's level is above the levels of all columns that update it; the update triplets
// of a level are exactly (L_rj, L_kj -> block (r, k)) for its columns j and every pair
// r >= k of j's rows, grouped into one task per destination; a near task is one whose
// destination column is factored at the next level.
void check_symbolic(const Topo& t, int order) {
  const int G = (int)t.height.size();
  float dummy[4] = {0, 0, 0, 0};
  int32_t midx[1] = {-1};
  como3r_graph_desc d{};
  d.num_graphs = G;
  d.kf_offset = t.kf_offset.data();
  d.height = t.height.data();
  d.width = t.width.data();
  d.agent_of = t.agent_of.data();
  d.points_conf = dummy;
  d.dtype = COMO3R_F32;
  d.edge_offset = t.edge_offset.data();
  d.edge_i = t.edge_i.data();
  d.edge_j = t.edge_j.data();
  d.match_idx = midx;
  d.anchor = t.anchor.data();
  d.sigma_ray = 0.003;
  d.sigma_dist = 10;
  d.huber_k = 1.345;
  d.eps0 = 1e-6;
  d.max_attempts = 6;
  d.mode = COMO3R_MIXED;
  HostPlan p;
  std::vector<int8_t> ord(G, (int8_t)order);
  CHECK(build_plan(&d, p, &ord) == COMO3R_OK, "%s: build_plan: %s", t.name.c_str(), p.error.c_str());
  for (int g = 0; g < G; ++g) {
    const int* m = p.meta.data() + kMetaCount * g;
    const int cbase = m[kMetaColBase], n = m[kMetaNCol], sbase = m[kMetaSlotBase], nslot = m[kMetaNSlot];
    const int nlev = m[kMetaNLvl], ubase = m[kMetaUBase], tribase = m[kMetaTriBase];
    const int* lvl = p.llvl.data() + 4 * m[kMetaLvlBase];
    const int* colslot = p.lcol_slot.data() + cbase + g;
    CHECK(colslot[n] == nslot, "%s: column slots end at %d, %d slots", t.name.c_str(), colslot[n], nslot);
    // columns <-> keyframes: every unfixed keyframe of the graph exactly once
    std::map<int, int> col_of_kf;
    for (int c = 0; c < n; ++c) {
      const int kf = p.col_kf[cbase + c];
      CHECK(kf >= t.kf_offset[g] && kf < t.kf_offset[g + 1] && !p.frozen[kf] && !col_of_kf.count(kf),
            "%s: column %d keyframe %d", t.name.c_str(), c, kf);
      col_of_kf[kf] = c;
    }
    int unfixed = 0;
    for (int kf = t.kf_offset[g]; kf < t.kf_offset[g + 1]; ++kf) unfixed += !p.frozen[kf];
    CHECK(unfixed == n, "%s: %d unfixed keyframes, %d columns", t.name.c_str(), unfixed, n);
    // elimination graph in column order
    std::vector<std::vector<char>> adj(n, std::vector<char>(n, 0));
    for (int e = t.edge_offset[g]; e < t.edge_offset[g + 1]; ++e) {
      const auto a = col_of_kf.find(t.edge_i[e]), b = col_of_kf.find(t.edge_j[e]);
      if (a == col_of_kf.end() || b == col_of_kf.end()) continue;
      adj[a->second][b->second] = adj[b->second][a->second] = 1;
    }
    std::vector<std::vector<int>> rows(n);
    for (int c = 0; c < n; ++c) {
      for (int r = c + 1; r < n; ++r)
        if (adj[c][r]) rows[c].push_back(r);
      for (int a : rows[c])
        for (int b : rows[c])
          if (a != b) adj[a][b] = 1;
    }
    std::map<std::pair<int, int>, int> slot;  // (row, column) -> local slot
    for (int c = 0; c < n; ++c) {
      const int s0 = colslot[c], nb = colslot[c + 1] - s0 - 1;
      CHECK(p.lslot_row[sbase + s0] == c, "%s: column %d's first slot is not its diagonal", t.name.c_str(), c);
      CHECK(nb == (int)rows[c].size(), "%s order %d: column %d has %d off-diagonal blocks, elimination gives %zu",
            t.name.c_str(), order, c, nb, rows[c].size());
      slot[{c, c}] = s0;
      for (int b = 0; b < nb; ++b) {
        CHECK(p.lslot_row[sbase + s0 + 1 + b] == rows[c][b], "%s order %d: column %d block %d row %d, expected %d",
              t.name.c_str(), order, c, b, p.lslot_row[sbase + s0 + 1 + b], rows[c][b]);
        slot[{rows[c][b], c}] = s0 + 1 + b;
      }
    }
    // levels
    std::vector<int> level(n, -1);
    for (int l = 0; l < nlev; ++l)
      for (int q = lvl[4 * l]; q < lvl[4 * (l + 1)]; ++q) {
        const int c = p.lsched[cbase + q];
        CHECK(c >= 0 && c < n && level[c] < 0, "%s: column %d scheduled twice", t.name.c_str(), c);
        level[c] = l;
      }
    for (int c = 0; c < n; ++c) {
      CHECK(level[c] >= 0, "%s: column %d never scheduled", t.name.c_str(), c);
      for (int r : rows[c])
        CHECK(level[r] > level[c], "%s: column %d (level %d) updates column %d at level %d", t.name.c_str(), c,
              level[c], r, level[r]);
    }
    // update triplets per level
    for (int l = 0; l < nlev; ++l) {
      std::map<std::vector<int>, int> want, got;
      for (int j = 0; j < n; ++j) {
        if (level[j] != l) continue;
        for (size_t a = 0; a < rows[j].size(); ++a)
          for (size_t b = 0; b <= a; ++b) {
            const int r = rows[j][a], k = rows[j][b];
            ++want[{slot[{r, j}], slot[{k, j}], slot[{r, k}], j}];
          }
      }
      for (int v = lvl[4 * l + 1]; v < lvl[4 * (l + 1) + 1]; ++v) {
        const int4 tk = p.lutask[ubase + v];
        const bool diag = p.lslot_row[sbase + tk.x] == [&] {
          for (int c = 0; c < n; ++c)
            if (tk.x >= colslot[c] && tk.x < colslot[c + 1]) return c;
          return -1;
        }();
        CHECK(tk.w == (diag ? p.lslot_row[sbase + tk.x] : -1), "%s: task of slot %d right-hand-side column %d",
              t.name.c_str(), tk.x, tk.w);
        int dst_col = -1;
        for (int c = 0; c < n; ++c)
          if (tk.x >= colslot[c] && tk.x < colslot[c + 1]) dst_col = c;
        const bool near = v < lvl[4 * l + 2];
        CHECK(near == (level[dst_col] == l + 1), "%s: task of slot %d (column level %d) near=%d at level %d",
              t.name.c_str(), tk.x, level[dst_col], (int)near, l);
        for (int q = tk.y; q < tk.z; ++q) {
          const int4 tr = p.ltri[tribase + q];
          CHECK(tr.z == tk.x, "%s: triplet of slot %d in the task of slot %d", t.name.c_str(), tr.z, tk.x);
          ++got[{tr.x, tr.y, tr.z, tr.w}];
        }
      }
      CHECK(want == got, "%s order %d level %d: %zu distinct update triplets planned, %zu expected", t.name.c_str(),
            order, l, got.size(), want.size());
    }
  }
}

// The CTA-group plan of a batch (build_group_plan): every graph exactly once; a clustered
// graph on kGroupCTAs consecutive CTAs of ranks 0..kGroupCTAs-1, the others packed onto
// single CTAs; whole clusters within the GPU; the clustered graphs the slowest by the
// one-CTA estimate; a forced count honoured.
void check_groups(const Topo& t, int sms) {
  const int G = (int)t.height.size();
  float dummy[4] = {0, 0, 0, 0};
  int32_t midx[1] = {-1};
  como3r_graph_desc d{};
  d.num_graphs = G;
  d.kf_offset = t.kf_offset.data();
  d.height = t.height.data();
  d.width = t.width.data();
  d.agent_of = t.agent_of.data();
  d.points_conf = dummy;
  d.dtype = COMO3R_F32;
  d.edge_offset = t.edge_offset.data();
  d.edge_i = t.edge_i.data();
  d.edge_j = t.edge_j.data();
  d.match_idx = midx;
  d.anchor = t.anchor.data();
  d.sigma_ray = 0.003;
  d.sigma_dist = 10;
  d.huber_k = 1.345;
  d.eps0 = 1e-6;
  d.max_attempts = 6;
  d.mode = COMO3R_MIXED;
  HostPlan p;
  CHECK(build_plan(&d, p) == COMO3R_OK, "%s: build_plan: %s", t.name.c_str(), p.error.c_str());
  for (int force : {-1, 1, 3}) {
    GroupPlan gp;
    build_group_plan(p, sms, force, gp);
    if (gp.ctas == 0) {
      CHECK(force < 0, "%s: forced %d clustered graphs, no group plan", t.name.c_str(), force);
      continue;
    }
    CHECK(gp.ctas % kGroupCTAs == 0 && gp.ctas <= sms, "%s: %d CTAs on %d SMs", t.name.c_str(), gp.ctas, sms);
    CHECK((int)gp.gtask.size() == gp.ctas, "%s: %zu tasks for %d CTAs", t.name.c_str(), gp.gtask.size(), gp.ctas);
    if (force > 0) CHECK(gp.big == force, "%s: forced %d, planned %d", t.name.c_str(), force, gp.big);
    std::vector<int> seen(G, 0), clustered(G, 0);
    for (int c = 0; c < gp.ctas; ++c) {
      const int4 k = gp.gtask[c];
      CHECK(k.x >= 0 && k.y >= 0 && k.x + k.y <= (int)gp.glist.size(), "%s: CTA %d list out of range",
            t.name.c_str(), c);
      if (k.w == kGroupCTAs) {
        CHECK(k.y == 1 && c % kGroupCTAs == k.z, "%s: CTA %d rank %d of a cluster-solved graph", t.name.c_str(), c,
              k.z);
        CHECK(gp.gtask[c - k.z].x == k.x, "%s: CTA %d not in its graph's cluster", t.name.c_str(), c);
        if (k.z == 0) ++seen[gp.glist[k.x]], clustered[gp.glist[k.x]] = 1;
      } else {
        CHECK(k.w == 1 && k.z == 0, "%s: CTA %d group size %d rank %d", t.name.c_str(), c, k.w, k.z);
        for (int q = 0; q < k.y; ++q) ++seen[gp.glist[k.x + q]];
      }
    }
    int nclustered = 0;
    for (int g = 0; g < G; ++g) {
      CHECK(seen[g] == 1, "%s: graph %d solved %d times", t.name.c_str(), g, seen[g]);
      nclustered += clustered[g];
      CHECK((gp.order[g] >= 0) == (clustered[g] == 1), "%s: graph %d ordering override", t.name.c_str(), g);
    }
    CHECK(nclustered == gp.big, "%s: %d clustered graphs, planned %d", t.name.c_str(), nclustered, gp.big);
    // the clustered graphs are the slowest by the one-CTA estimate (levels and block updates
    // of the cheaper ordering for one SM): none of the others is estimated slower
    auto est = [&](int g) {
      const double md = 3.0 * p.nlev_md[g] + 0.15 * (double)p.upd_md[g];
      const double nd = 3.0 * p.nlev_nd[g] + 0.15 * (double)p.upd_nd[g];
      return md <= nd ? 6.3 * p.nlev_md[g] + 0.26 * (double)p.upd_md[g] : 6.3 * p.nlev_nd[g] + 0.26 * (double)p.upd_nd[g];
    };
    double min_big = 1e300, max_small = -1;
    for (int g = 0; g < G; ++g) {
      if (clustered[g]) min_big = std::min(min_big, est(g));
      else max_small = std::max(max_small, est(g));
    }
    CHECK(max_small <= min_big, "%s: a single-CTA graph (%.1f us) estimated slower than a clustered one (%.1f us)",
          t.name.c_str(), max_small, min_big);
  }
}

}  // namespace

int main() {
  std::vector<Topo> topos;
  {
    Topo t{"two_agents_40"};
    t.kf_offset = {0};
    t.edge_offset = {0};
    add_graph(t, 2, 40, 10, 6, 7u);
    topos.push_back(t);
  }
  {
    Topo t{"four_agents_150"};
    t.kf_offset = {0};
    t.edge_offset = {0};
    add_graph(t, 4, 150, 0, 60, 11u);
    topos.push_back(t);
  }
  {
    Topo t{"chain_400"};
    t.kf_offset = {0};
    t.edge_offset = {0};
    add_graph(t, 1, 400, 50, 0, 3u);
    topos.push_back(t);
  }
  {
    Topo t{"batch_3"};
    t.kf_offset = {0};
    t.edge_offset = {0};
    add_graph(t, 2, 12, 4, 2, 5u);
    add_graph(t, 3, 30, 10, 8, 9u);
    add_graph(t, 1, 60, 20, 0, 13u);
    topos.push_back(t);
  }
  for (const Topo& t : topos) {
    check_topology(t);
    check_symbolic(t, 0);
    check_symbolic(t, 1);
  }
  {
    Topo t{"batch_40"};
    t.kf_offset = {0};
    t.edge_offset = {0};
    for (int g = 0; g < 40; ++g) add_graph(t, 2, 6 + (g * 37) % 110, (g % 3) ? 10 : 0, 2 + g % 7, 100u + g);
    check_groups(t, 148);
    check_groups(t, 64);
  }
  std::printf("OK %d\n", g_checks);
  return 0;
}
