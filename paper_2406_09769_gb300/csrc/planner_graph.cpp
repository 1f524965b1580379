// Host-side planner of Algorithm partitioned_contract (Sec. 3.2) for any
// closed graph and any partition, on the maximally unbalanced path of the
// paper's lattice and random-regular-graph experiments (Sec. 7.3).
//
// Per contraction (I_{s-1} with V_s; the first joins V_0 and V_1):
//   * edge sets E(V_a, V_b) between parts (Algorithm partitioned_contract),
//     each ordered by (vertex in the earlier part, vertex in the later part,
//     edge id);
//   * the reference ordering tau_s of the open edge sets: sigma_{s-1} with the
//     sets into V_s replaced, where the first of them stood, by V_s's own
//     sets (ordered by the later part); tau_1 lists V_1's sets by later part;
//   * the constraint tree of the parts still to come (the appendix on the
//     constraint tree): node i joins the sets into the i-th next part with
//     the subtrees of earlier nodes whose parts are adjacent to it;
//   * sigma_s = Algorithm linear_ordering_under_constraint_tree: every node's
//     children in the order whose concatenation has the least Kendall-Tau
//     distance to tau_s (exact subset programme up to 12 children, ties to
//     the lexicographically first order; beyond, by mean tau position);
//   * Algorithm approx_tensor_network: d = Kendall-Tau distance(tau_s,
//     sigma_s), ceil(d / r) density-matrix passes at the orderings r swaps
//     apart on the bubble-sort path from tau_s to sigma_s (r <= 0: one pass);
//   * per pass, the MPS embedding tree (App. C) over the leaves and the
//     embedding phi of the network's tensors along its chain (Algorithm
//     tree_embedding: at every tree edge the inclusion-minimal minimum cut
//     between the leaves on its two sides, weights round(2^16 log2 dim);
//     these cuts are nested, so each tensor sits at the first cut whose
//     source side holds it);
//   * the block of every chain position: its tensors contracted together
//     ("contract T(v) first", Sec. 5.3) with a delta for every edge passing
//     through, legs (edges crossing the left cut, leaf, edges crossing the
//     right cut), crossing edges ordered by (MPS bond before graph edge, id).
// The last contraction closes the network along the chain of the final MPS.
// An intermediate with fewer than 3 open edges absorbs the next part too.
#include <algorithm>
#include <array>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <functional>
#include <map>
#include <set>
#include <string>
#include <utility>
#include <vector>

#include "tn_internal.h"

namespace tn {

namespace {

[[noreturn]] void fail(tn_status st, const std::string& m) { throw PlanFail{st, m}; }

// An edge label of the network of one contraction: kind 0 = bond k of the
// current MPS, kind 1 = graph edge e.  Ordered by (kind, id).
struct Lab {
  int32_t kind, id;
  bool operator<(const Lab& o) const { return kind != o.kind ? kind < o.kind : id < o.id; }
  bool operator==(const Lab& o) const { return kind == o.kind && id == o.id; }
};
// A tensor of that network: kind 0 = MPS site k, kind 1 = graph vertex v.
struct Ten {
  int32_t kind, id;
  std::vector<Lab> legs;
};

using SetKey = std::pair<int32_t, int32_t>;  // (earlier part a, later part b)

int64_t capacity(int64_t dim) { return llround(65536.0 * std::log2(double(dim))); }

int64_t kt_distance(const std::vector<SetKey>& a, const std::vector<SetKey>& b) {
  std::map<SetKey, int> pos;
  for (size_t i = 0; i < b.size(); ++i) pos[b[i]] = int(i);
  std::vector<int> seq;
  for (const SetKey& k : a) seq.push_back(pos.at(k));
  int64_t d = 0;
  for (size_t i = 0; i < seq.size(); ++i)
    for (size_t j = i + 1; j < seq.size(); ++j)
      if (seq[i] > seq[j]) ++d;
  return d;
}

// Order of the children (each a fixed list of sets) whose concatenation has
// the least Kendall-Tau distance to tau (tau_pos: position of every set).
std::vector<int> best_permutation(const std::vector<std::vector<SetKey>>& ch,
                                  const std::map<SetKey, int>& tau_pos) {
  const int m = int(ch.size());
  std::vector<int> order(m);
  for (int i = 0; i < m; ++i) order[i] = i;
  if (m <= 1) return order;
  std::vector<std::vector<int64_t>> cross(m, std::vector<int64_t>(m, 0));
  for (int x = 0; x < m; ++x)
    for (int y = 0; y < m; ++y) {
      if (x == y) continue;
      int64_t c = 0;
      for (const SetKey& e : ch[x])
        for (const SetKey& f : ch[y])
          if (tau_pos.at(f) < tau_pos.at(e)) ++c;
      cross[x][y] = c;
    }
  if (m > 12) {
    std::vector<int64_t> sum(m, 0);
    for (int x = 0; x < m; ++x)
      for (const SetKey& e : ch[x]) sum[x] += tau_pos.at(e);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
      const int64_t l = sum[x] * int64_t(ch[y].size()), r = sum[y] * int64_t(ch[x].size());
      if (l != r) return l < r;
      return x < y;
    });
    return order;
  }
  const int full = (1 << m) - 1;
  std::vector<int64_t> g(size_t(1) << m, 0);
  auto step_cost = [&](int S, int x) {
    const int rest = full & ~S & ~(1 << x);
    int64_t c = 0;
    for (int y = 0; y < m; ++y)
      if (rest >> y & 1) c += cross[x][y];
    return c + g[S | (1 << x)];
  };
  for (int S = full - 1; S >= 0; --S) {
    int64_t best = INT64_MAX;
    for (int x = 0; x < m; ++x)
      if (!(S >> x & 1)) best = std::min(best, step_cost(S, x));
    g[S] = best;
  }
  order.clear();
  int S = 0;
  while (S != full) {
    for (int x = 0; x < m; ++x) {
      if (S >> x & 1) continue;
      if (step_cost(S, x) == g[S]) {
        order.push_back(x);
        S |= 1 << x;
        break;
      }
    }
  }
  return order;
}

// Inclusion-minimal source side of a minimum cut between the terminal sets
// (nodes reachable from the sources in the residual graph of a maximum flow,
// Edmonds-Karp).  arcs: undirected (a, b, capacity).
std::vector<char> min_cut_source_side(int n_nodes, const std::vector<std::array<int64_t, 3>>& arcs,
                                      const std::vector<int>& src, const std::vector<int>& snk) {
  const int64_t INF = int64_t(1) << 60;
  const int s = n_nodes, t = n_nodes + 1, N = n_nodes + 2;
  struct Arc {
    int to, rev;
    int64_t cap;
  };
  std::vector<std::vector<Arc>> adj(N);
  auto add = [&](int a, int b, int64_t ca, int64_t cb) {
    adj[a].push_back({b, int(adj[b].size()), ca});
    adj[b].push_back({a, int(adj[a].size()) - 1, cb});
  };
  for (const auto& e : arcs) add(int(e[0]), int(e[1]), e[2], e[2]);
  for (int x : src) add(s, x, INF, 0);
  for (int x : snk) add(x, t, INF, 0);
  std::vector<int> pv(N), pa(N);
  std::vector<char> seen(N);
  std::vector<int> queue;
  queue.reserve(N);
  while (true) {
    std::fill(seen.begin(), seen.end(), 0);
    queue.clear();
    queue.push_back(s);
    seen[s] = 1;
    for (size_t h = 0; h < queue.size() && !seen[t]; ++h) {
      const int x = queue[h];
      for (int i = 0; i < int(adj[x].size()); ++i) {
        const Arc& a = adj[x][i];
        if (!seen[a.to] && a.cap > 0) {
          seen[a.to] = 1;
          pv[a.to] = x;
          pa[a.to] = i;
          queue.push_back(a.to);
        }
      }
    }
    if (!seen[t]) return std::vector<char>(seen.begin(), seen.begin() + n_nodes);
    int64_t f = INF;
    for (int y = t; y != s; y = pv[y]) f = std::min(f, adj[pv[y]][pa[y]].cap);
    for (int y = t; y != s; y = pv[y]) {
      Arc& a = adj[pv[y]][pa[y]];
      a.cap -= f;
      adj[y][a.rev].cap += f;
    }
  }
}

// ------------------------------------------------------------ edge orders

std::vector<SetKey> constraint_order(const std::vector<SetKey>& tau, int s, int N,
                                     const std::vector<std::set<int>>& adj_parts) {
  const int L = int(tau.size());
  std::map<SetKey, int> tau_pos;
  for (int p = 0; p < L; ++p) tau_pos[tau[p]] = p;
  std::vector<int> parent(L, -1);
  std::vector<std::vector<int>> children;
  std::vector<int> rep(std::max(N - s, 1), -1);
  auto top = [&](int x) {
    while (parent[x] >= 0) x = parent[x];
    return x;
  };
  auto new_node = [&](const std::vector<int>& kids) {
    const int node = L + int(children.size());
    children.push_back(kids);
    parent.push_back(-1);
    for (int x : kids) parent[x] = node;
    return node;
  };
  for (int i = 1; i < N - s; ++i) {
    const int b = s + i;
    std::vector<int> kids;
    for (int p = 0; p < L; ++p)
      if (tau[p].second == b) kids.push_back(p);
    for (int j = 1; j < i; ++j)
      if (adj_parts[b].count(s + j) && rep[j] >= 0) kids.push_back(top(rep[j]));
    std::vector<int> uniq;
    for (int x : kids)
      if (std::find(uniq.begin(), uniq.end(), x) == uniq.end()) uniq.push_back(x);
    if (uniq.size() >= 2)
      rep[i] = new_node(uniq);
    else if (uniq.size() == 1)
      rep[i] = uniq[0];
    else
      rep[i] = -1;
  }
  std::vector<int> roots;
  for (int p = 0; p < L; ++p) {
    const int t = top(p);
    if (std::find(roots.begin(), roots.end(), t) == roots.end()) roots.push_back(t);
  }
  const int root = roots.size() == 1 ? roots[0] : new_node(roots);
  std::function<std::vector<SetKey>(int)> order_of = [&](int x) -> std::vector<SetKey> {
    if (x < L) return {tau[x]};
    std::vector<std::vector<SetKey>> subs;
    for (int c : children[x - L]) subs.push_back(order_of(c));
    auto first = [&](const std::vector<SetKey>& o) {
      int m = INT_MAX;
      for (const SetKey& k : o) m = std::min(m, tau_pos.at(k));
      return m;
    };
    std::stable_sort(subs.begin(), subs.end(),
                     [&](const std::vector<SetKey>& u, const std::vector<SetKey>& v) {
                       return first(u) < first(v);
                     });
    std::vector<SetKey> out;
    for (int q : best_permutation(subs, tau_pos))
      out.insert(out.end(), subs[q].begin(), subs[q].end());
    return out;
  };
  return order_of(root);
}

std::vector<std::vector<SetKey>> swap_path(const std::vector<SetKey>& tau,
                                           const std::vector<SetKey>& sigma, int64_t r,
                                           int64_t n_pass) {
  std::map<SetKey, int> rank;
  for (size_t i = 0; i < sigma.size(); ++i) rank[sigma[i]] = int(i);
  std::vector<SetKey> seq(tau);
  std::vector<std::vector<SetKey>> snaps{seq};
  bool changed = true;
  while (changed) {
    changed = false;
    for (size_t i = 0; i + 1 < seq.size(); ++i)
      if (rank[seq[i]] > rank[seq[i + 1]]) {
        std::swap(seq[i], seq[i + 1]);
        snaps.push_back(seq);
        changed = true;
      }
  }
  const int64_t d = int64_t(snaps.size()) - 1;
  std::vector<std::vector<SetKey>> out;
  for (int64_t p = 1; p <= n_pass; ++p) out.push_back(snaps[size_t(std::min(p * r, d))]);
  return out;
}

// ---------------------------------------------------------- chain layout

constexpr int64_t kMaxCut = 4096;  // largest untruncated tree-edge dim planned

struct Layout {
  std::vector<int> phi;
  std::vector<std::vector<Lab>> cross;
  std::vector<int32_t> D;
};

Layout chain_layout(const std::vector<Ten>& T, const std::map<Lab, int64_t>& dim,
                    const std::vector<Lab>& leaves, int n_pos) {
  const int nt = int(T.size());
  std::map<Lab, std::vector<int>> where;
  for (int i = 0; i < nt; ++i)
    for (const Lab& l : T[i].legs) where[l].push_back(i);
  std::vector<std::array<int64_t, 3>> arcs;
  for (const auto& kv : where) {
    if (kv.second.size() > 2) fail(TN_ERR_INVALID, "an edge joins more than two tensors");
    if (kv.second.size() == 2)
      arcs.push_back({kv.second[0], kv.second[1], capacity(dim.at(kv.first))});
  }
  std::map<Lab, int> pi;
  std::vector<int> term;
  int n_nodes = nt;
  if (!leaves.empty()) {
    for (int j = 0; j < int(leaves.size()); ++j) {
      const auto it = where.find(leaves[j]);
      if (it == where.end() || it->second.size() != 1) fail(TN_ERR_INVALID, "leaf without one owner");
      pi[leaves[j]] = j;
      arcs.push_back({it->second[0], nt + j, capacity(dim.at(leaves[j]))});
      term.push_back(nt + j);
    }
    n_nodes = nt + int(leaves.size());
  } else {
    for (int k = 0; k < n_pos; ++k) term.push_back(k);  // MPS sites come first
  }
  for (const auto& kv : where)
    if (kv.second.size() == 1 && !pi.count(kv.first)) fail(TN_ERR_INVALID, "dangling edge");
  Layout L;
  L.phi.assign(nt, -1);
  for (int k = 0; k + 1 < n_pos; ++k) {
    std::vector<int> src(term.begin(), term.begin() + k + 1), snk(term.begin() + k + 1, term.end());
    const std::vector<char> left = min_cut_source_side(n_nodes, arcs, src, snk);
    for (int i = 0; i < nt; ++i)
      if (L.phi[i] < 0 && left[i]) L.phi[i] = k;
  }
  for (int i = 0; i < nt; ++i)
    if (L.phi[i] < 0) L.phi[i] = n_pos - 1;
  L.cross.assign(std::max(n_pos - 1, 0), {});
  for (const auto& kv : where) {
    int a, b;
    if (kv.second.size() == 2) {
      a = L.phi[kv.second[0]];
      b = L.phi[kv.second[1]];
    } else {
      a = L.phi[kv.second[0]];
      b = pi.at(kv.first);
    }
    for (int k = std::min(a, b); k < std::max(a, b); ++k) L.cross[k].push_back(kv.first);
  }
  L.D.assign(n_pos, 1);
  for (int k = 0; k + 1 < n_pos; ++k) {
    std::sort(L.cross[k].begin(), L.cross[k].end());
    int64_t D = 1;
    for (const Lab& l : L.cross[k]) {
      D *= dim.at(l);
      if (D > kMaxCut) fail(TN_ERR_UNSUPPORTED, "an untruncated tree edge exceeds 4096");
    }
    L.D[k] = int32_t(D);
  }
  return L;
}

// Op programs of every chain position (see GOpH / GTensorH).
constexpr int64_t kMaxScratch = int64_t(1) << 22;  // elements of one intermediate

void block_programs(Step& st, const std::vector<Ten>& T, const std::map<Lab, int64_t>& dim,
                    const std::vector<Lab>& leaves, const Layout& L, int n_pos) {
  struct Operand {
    std::vector<Lab> labs;  // memory order (row-major, the first slowest)
    int32_t src, id, level;
  };
  std::vector<GOpH> ops;
  std::vector<std::vector<GTensorH>> op_ten;
  std::vector<std::vector<std::vector<std::pair<int32_t, int32_t>>>> op_legs;
  std::vector<std::vector<int32_t>> op_code;
  int64_t scratch = 0;
  auto size_of = [&](const std::vector<Lab>& ls) {
    int64_t s = 1;
    for (const Lab& l : ls) s *= dim.at(l);
    return s;
  };
  // emits one op: operands ins, output labels outs (a label listed twice is a
  // delta), every other label of the operands summed
  auto emit = [&](int k, const std::vector<Operand>& ins, const std::vector<Lab>& outs,
                  bool to_block) {
    std::vector<Lab> slots;
    auto slot_of = [&](const Lab& l) {
      for (size_t i = 0; i < slots.size(); ++i)
        if (slots[i] == l) return int32_t(i);
      slots.push_back(l);
      return int32_t(slots.size()) - 1;
    };
    std::vector<int32_t> os;
    for (const Lab& l : outs) os.push_back(slot_of(l));
    const int n_out = int(slots.size());
    std::vector<GTensorH> ten;
    std::vector<std::vector<std::pair<int32_t, int32_t>>> legs;
    int level = 0;
    for (const Operand& o : ins) {
      std::vector<std::pair<int32_t, int32_t>> lg(o.labs.size());
      int64_t stride = 1;
      for (int j = int(o.labs.size()) - 1; j >= 0; --j) {
        lg[j] = {slot_of(o.labs[j]), int32_t(stride)};
        stride *= dim.at(o.labs[j]);
      }
      if (stride >= (int64_t(1) << 31)) fail(TN_ERR_UNSUPPORTED, "tensor too large");
      GTensorH g{};
      g.src = o.src;
      g.id = o.id;
      g.nleg = int32_t(lg.size());
      ten.push_back(g);
      legs.push_back(lg);
      level = std::max(level, o.level + 1);
    }
    GOpH op{};
    op.pos = k;
    op.level = level;
    op.to_block = to_block ? 1 : 0;
    op.ns = int32_t(slots.size());
    op.nout = int32_t(os.size());
    op.nsum = op.ns - n_out;
    op.nt = int32_t(ten.size());
    if (op.ns > 48 || op.nout > 32 || op.nsum > 16 || op.nt > 8)
      fail(TN_ERR_UNSUPPORTED, "block op with too many edges");
    int64_t ne = 1;
    for (int32_t s : os) ne *= dim.at(slots[s]);
    op.n_elems = ne;
    if (!to_block) {
      if (ne > kMaxScratch) fail(TN_ERR_UNSUPPORTED, "block intermediate too large");
      op.dst_off = scratch;
      scratch += ne;
    }
    std::vector<int32_t> code;
    for (const Lab& l : slots) code.push_back(int32_t(dim.at(l)));
    code.insert(code.end(), os.begin(), os.end());
    for (int i = n_out; i < op.ns; ++i) code.push_back(i);
    ops.push_back(op);
    op_ten.push_back(ten);
    op_legs.push_back(legs);
    op_code.push_back(code);
    return int(ops.size()) - 1;
  };
  for (int k = 0; k < n_pos; ++k) {
    static const std::vector<Lab> none;
    const std::vector<Lab>& left = k >= 1 ? L.cross[k - 1] : none;
    const std::vector<Lab>& right = k + 1 < n_pos ? L.cross[k] : none;
    std::vector<Lab> outs(left);
    if (!leaves.empty()) outs.push_back(leaves[k]);
    outs.insert(outs.end(), right.begin(), right.end());
    std::set<Lab> out_set(outs.begin(), outs.end());
    std::vector<Operand> cur;
    for (int i = 0; i < int(T.size()); ++i)
      if (L.phi[i] == k) cur.push_back({T[i].legs, T[i].kind == 0 ? 1 : 0, T[i].id, -1});
    // greedy pairwise contraction: the smallest result first, then the least
    // work, then the first pair
    while (cur.size() > 1) {
      std::map<Lab, int> count;
      for (const Operand& o : cur)
        for (const Lab& l : o.labs) count[l]++;
      int bi = -1, bj = -1;
      bool b_share = false;
      int64_t b_size = 0, b_work = 0;
      std::vector<Lab> b_res, b_sum;
      for (int i = 0; i < int(cur.size()); ++i)
        for (int j = i + 1; j < int(cur.size()); ++j) {
          std::vector<Lab> res, sum;
          for (const Lab& l : cur[i].labs) {
            const bool shared = std::find(cur[j].labs.begin(), cur[j].labs.end(), l) != cur[j].labs.end();
            if (shared && !out_set.count(l) && count[l] == 2)
              sum.push_back(l);
            else
              res.push_back(l);
          }
          for (const Lab& l : cur[j].labs)
            if (std::find(sum.begin(), sum.end(), l) == sum.end() &&
                std::find(res.begin(), res.end(), l) == res.end())
              res.push_back(l);
          const bool share = !sum.empty();
          const int64_t sz = size_of(res), wk = sz * size_of(sum);
          const bool better = bi < 0 || (share && !b_share) ||
                              (share == b_share && (sz < b_size || (sz == b_size && wk < b_work)));
          if (better) {
            bi = i; bj = j; b_share = share; b_size = sz; b_work = wk;
            b_res = res; b_sum = sum;
          }
        }
      const int id = emit(k, {cur[bi], cur[bj]}, b_res, false);
      Operand r{b_res, 2, int32_t(ops[id].dst_off), ops[id].level};
      cur.erase(cur.begin() + bj);
      cur.erase(cur.begin() + bi);
      cur.push_back(r);
    }
    const int fid = emit(k, cur, outs, true);
    GOpH& f = ops[fid];
    f.Dl = k >= 1 ? L.D[k - 1] : 1;
    f.dkDr = int32_t(f.n_elems / f.Dl);
    if (f.n_elems != int64_t(f.Dl) * (leaves.empty() ? 1 : dim.at(leaves[k])) * L.D[k])
      fail(TN_ERR_INVALID, "block shape mismatch");
  }
  // order by level, then lay out operands and code
  std::vector<int> order(ops.size());
  for (size_t i = 0; i < ops.size(); ++i) order[i] = int(i);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return ops[x].level < ops[y].level; });
  st.gop.clear();
  st.gten.clear();
  st.gcode.clear();
  int max_level = -1;
  for (int i : order) {
    GOpH op = ops[i];
    op.code_off = int32_t(st.gcode.size());
    st.gcode.insert(st.gcode.end(), op_code[i].begin(), op_code[i].end());
    op.t_first = int32_t(st.gten.size());
    for (size_t t = 0; t < op_ten[i].size(); ++t) {
      GTensorH g = op_ten[i][t];
      g.leg_off = int32_t(st.gcode.size());
      for (const auto& pr : op_legs[i][t]) {
        st.gcode.push_back(pr.first);
        st.gcode.push_back(pr.second);
      }
      st.gten.push_back(g);
    }
    max_level = std::max(max_level, op.level);
    st.gop.push_back(op);
  }
  st.level_start.assign(max_level + 2, 0);
  for (const GOpH& op : st.gop) st.level_start[op.level + 1]++;
  for (int j = 0; j <= max_level; ++j) st.level_start[j + 1] += st.level_start[j];
  st.scratch_elems = scratch;
}

}  // namespace

void build_general_steps(const tn_graph* g, const tn_plan_opts* o,
                         std::vector<std::vector<int>> parts, tn_plan_t* P) {
  const int nv = g->n_vertices, ne = g->n_edges;
  for (auto& p : parts) std::sort(p.begin(), p.end());
  // an intermediate with fewer than 3 open edges absorbs the next part too
  {
    std::vector<char> inside(nv, 0);
    size_t s = 1;
    while (s + 2 <= parts.size()) {
      std::fill(inside.begin(), inside.end(), 0);
      for (size_t i = 0; i <= s; ++i)
        for (int v : parts[i]) inside[v] = 1;
      int n_open = 0;
      for (int e = 0; e < ne; ++e)
        if (inside[g->edge_u[e]] != inside[g->edge_v[e]]) ++n_open;
      if (n_open < 3) {
        parts[s].insert(parts[s].end(), parts[s + 1].begin(), parts[s + 1].end());
        std::sort(parts[s].begin(), parts[s].end());
        parts.erase(parts.begin() + s + 1);
      } else {
        ++s;
      }
    }
  }
  const int N = int(parts.size());
  if (N < 3) fail(TN_ERR_UNSUPPORTED, "need at least one approximated intermediate");
  P->n_contractions = N - 1;
  std::vector<int> part_of(nv, -1);
  for (int i = 0; i < N; ++i)
    for (int v : parts[i]) part_of[v] = i;
  std::map<SetKey, std::vector<int>> sets;
  std::vector<std::set<int>> adj_parts(N);
  for (int e = 0; e < ne; ++e) {
    int a = part_of[g->edge_u[e]], b = part_of[g->edge_v[e]];
    if (a == b) continue;
    if (a > b) std::swap(a, b);
    sets[{a, b}].push_back(e);
    adj_parts[a].insert(b);
    adj_parts[b].insert(a);
  }
  auto in_part = [&](int e, int p) {
    return part_of[g->edge_u[e]] == p ? g->edge_u[e] : g->edge_v[e];
  };
  for (auto& kv : sets) {
    const int a = kv.first.first, b = kv.first.second;
    std::sort(kv.second.begin(), kv.second.end(), [&](int x, int y) {
      const int ax = in_part(x, a), ay = in_part(y, a);
      if (ax != ay) return ax < ay;
      const int bx = in_part(x, b), by = in_part(y, b);
      if (bx != by) return bx < by;
      return x < y;
    });
  }
  auto expand = [&](const std::vector<SetKey>& order) {
    std::vector<Lab> out;
    for (const SetKey& k : order)
      for (int e : sets.at(k)) out.push_back({1, e});
    return out;
  };
  std::vector<std::vector<int>> inc(nv);
  for (int e = 0; e < ne; ++e) {
    inc[g->edge_u[e]].push_back(e);
    inc[g->edge_v[e]].push_back(e);
  }
  for (auto& l : inc) std::sort(l.begin(), l.end());
  std::map<Lab, int64_t> dim;
  for (int e = 0; e < ne; ++e) dim[{1, e}] = g->edge_dim[e];
  std::vector<SetKey> sigma;
  for (const auto& kv : sets)
    if (kv.first.first == 0) sigma.push_back(kv.first);
  std::stable_sort(sigma.begin(), sigma.end(),
                   [](const SetKey& x, const SetKey& y) { return x.second < y.second; });
  std::vector<Lab> mps_leaves;
  std::vector<int32_t> mps_bonds;
  bool have_mps = false;
  auto site_tensors = [&](const std::vector<Lab>& leaves) {
    std::vector<Ten> T;
    const int m = int(leaves.size());
    for (int k = 0; k < m; ++k) {
      Ten t{0, k, {}};
      if (k >= 1) t.legs.push_back({0, k - 1});
      t.legs.push_back(leaves[k]);
      if (k <= m - 2) t.legs.push_back({0, k});
      T.push_back(t);
    }
    return T;
  };
  auto fill_sites = [](Step& st) {
    st.site.assign(st.n, SiteOp{});
    for (int k = 0; k < st.n; ++k) {
      SiteOp& op = st.site[k];
      op.vertex = -1;
      op.dp = op.dhl = op.dhr = 1;
      op.de = st.d[k];
      op.a = k >= 1 ? st.D[k - 1] : 1;
      op.b = st.D[k];
    }
  };
  for (int s = 1; s < N; ++s) {
    std::vector<int> raw = (s == 1) ? parts[0] : parts[s];
    if (s == 1) raw.insert(raw.end(), parts[1].begin(), parts[1].end());
    std::sort(raw.begin(), raw.end());
    std::vector<Ten> T;
    if (have_mps) {
      T = site_tensors(mps_leaves);
      for (size_t k = 0; k < mps_bonds.size(); ++k) dim[{0, int32_t(k)}] = mps_bonds[k];
    }
    for (int v : raw) {
      Ten t{1, v, {}};
      for (int e : inc[v]) t.legs.push_back({1, e});
      T.push_back(t);
    }
    if (s == N - 1) {
      const int m = int(mps_leaves.size());
      const Layout L = chain_layout(T, dim, {}, m);
      Step st;
      st.kind = 2;
      st.general = true;
      st.n = m;
      st.d.assign(m, 1);
      st.D = L.D;
      fill_sites(st);
      block_programs(st, T, dim, {}, L, m);
      step_layouts(st);
      P->steps.push_back(std::move(st));
      break;
    }
    std::vector<SetKey> kept, fresh;
    int at = -1;
    for (size_t i = 0; i < sigma.size(); ++i) {
      if (sigma[i].second == s) {
        if (at < 0) at = int(kept.size());
      } else {
        kept.push_back(sigma[i]);
      }
    }
    for (const auto& kv : sets)
      if (kv.first.first == s) fresh.push_back(kv.first);
    std::stable_sort(fresh.begin(), fresh.end(),
                     [](const SetKey& x, const SetKey& y) { return x.second < y.second; });
    if (at < 0) at = int(kept.size());
    std::vector<SetKey> tau(kept.begin(), kept.begin() + at);
    tau.insert(tau.end(), fresh.begin(), fresh.end());
    tau.insert(tau.end(), kept.begin() + at, kept.end());
    const std::vector<SetKey> sig = constraint_order(tau, s, N, adj_parts);
    const int64_t d_kt = kt_distance(tau, sig);
    std::vector<std::vector<SetKey>> orders;
    if (o->swap_batch > 0) {
      const int64_t n_pass = std::max<int64_t>(1, (d_kt + o->swap_batch - 1) / o->swap_batch);
      orders = swap_path(tau, sig, o->swap_batch, n_pass);
    } else {
      orders.push_back(sig);
    }
    for (const auto& order : orders) {
      const std::vector<Lab> leaves = expand(order);
      const int nl = int(leaves.size());
      if (nl < 3) fail(TN_ERR_UNSUPPORTED, "intermediates need >= 3 open legs");
      const Layout L = chain_layout(T, dim, leaves, nl);
      Step st;
      st.kind = 1;
      st.general = true;
      st.n = nl;
      st.n_kt = int32_t(d_kt);
      for (const Lab& l : leaves) {
        st.d.push_back(int32_t(dim.at(l)));
        st.leaves.push_back(l.id);
      }
      st.D = L.D;
      st.r.assign(nl - 1, 0);
      st.r[0] = st.d[0];
      for (int k = 1; k <= nl - 2; ++k) {
        int64_t beyond = 1;
        for (int j = k + 1; j < nl; ++j) beyond = std::min<int64_t>(beyond * st.d[j], int64_t(1) << 40);
        int64_t r = std::min<int64_t>(o->chi_max, int64_t(st.r[k - 1]) * st.d[k]);
        r = std::min<int64_t>(r, st.D[k]);
        r = std::min<int64_t>(r, beyond);
        st.r[k] = int32_t(r);
      }
      fill_sites(st);
      block_programs(st, T, dim, leaves, L, nl);
      step_layouts(st);
      // the next pass sees only the MPS this pass writes
      mps_leaves = leaves;
      mps_bonds.assign(st.r.begin(), st.r.end());
      have_mps = true;
      T = site_tensors(mps_leaves);
      for (size_t k = 0; k < mps_bonds.size(); ++k) dim[{0, int32_t(k)}] = mps_bonds[k];
      P->steps.push_back(std::move(st));
    }
    sigma = sig;
  }
}

}  // namespace tn
