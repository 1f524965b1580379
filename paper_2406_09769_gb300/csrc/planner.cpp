// Host-side planner of Algorithm partitioned_contract (Sec. 3.2).
//
// Builds, from the graph alone (never tensor data, Sec. 3.2), the sequence of
// contractions on a maximally unbalanced path over the parts, the MPS
// embedding tree of every intermediate (App. C, Def. MPS tree / MPS embedding
// tree), the embedding phi of its tensors (the boundary site and the part
// vertex aligned with leaf k go to the tree vertex of leaf k) and the shapes of
// every block, density matrix and output tensor, with flop counts from the
// cost model of Sec. 2.2.
//
// Supported structure ("boundary absorption"): every part is a simple path
// u_0 .. u_{m-1}; for every part after the first, u_i absorbs exactly the i-th
// open leg of the intermediate; every vertex of a non-final part emits exactly
// one new open leg, which takes the place of the absorbed one.  For such
// intermediates the edge-set ordering equals the reference ordering, so the
// Kendall-Tau distance of Algorithm approx_tensor_network is 0 and one
// density_matrix_alg pass runs per contraction (Sec. 6).
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "tn_internal.h"

namespace tn {

static thread_local std::string g_err;
void set_error(const std::string& msg) { g_err = msg; }
const char* get_error() { return g_err.c_str(); }

static bool same_ops(const SiteOp& x, const SiteOp& y) {
  return x.vertex == y.vertex && x.t_off == y.t_off && x.dp == y.dp && x.dhl == y.dhl &&
         x.dhr == y.dhr && x.de == y.de && x.sp == y.sp && x.shl == y.shl && x.shr == y.shr &&
         x.se == y.se && x.a == y.a && x.b == y.b;
}

bool plans_equivalent(const tn_plan_t* a, const tn_plan_t* b) {
  if (a == b) return true;
  if (a->n_vertices != b->n_vertices || a->chi != b->chi || a->site_elems != b->site_elems ||
      a->steps.size() != b->steps.size() || a->site_off != b->site_off)
    return false;
  for (size_t s = 0; s < a->steps.size(); ++s) {
    const Step& x = a->steps[s];
    const Step& y = b->steps[s];
    if (x.kind != y.kind || x.n != y.n || x.d != y.d || x.D != y.D || x.r != y.r ||
        x.general != y.general)
      return false;
    for (int k = 0; k < x.n; ++k)
      if (!same_ops(x.site[k], y.site[k])) return false;
    if (x.general) {
      if (x.gcode != y.gcode || x.gten.size() != y.gten.size() || x.gop.size() != y.gop.size() ||
          x.level_start != y.level_start || x.scratch_elems != y.scratch_elems)
        return false;
      for (size_t i = 0; i < x.gop.size(); ++i) {
        const GOpH &p = x.gop[i], &q = y.gop[i];
        if (p.pos != q.pos || p.level != q.level || p.to_block != q.to_block ||
            p.dst_off != q.dst_off || p.n_elems != q.n_elems || p.Dl != q.Dl ||
            p.dkDr != q.dkDr || p.ns != q.ns || p.nout != q.nout || p.nsum != q.nsum ||
            p.nt != q.nt || p.t_first != q.t_first || p.code_off != q.code_off)
          return false;
      }
      for (size_t i = 0; i < x.gten.size(); ++i) {
        const GTensorH &p = x.gten[i], &q = y.gten[i];
        if (p.src != q.src || p.id != q.id || p.nleg != q.nleg || p.leg_off != q.leg_off)
          return false;
      }
    }
  }
  return true;
}

}  // namespace tn

using tn::set_error;

namespace {

using Fail = tn::PlanFail;

[[noreturn]] void fail(tn_status st, const std::string& msg) { throw Fail{st, msg}; }

int64_t cap_mul(int64_t a, int64_t b) {
  const int64_t CAP = int64_t(1) << 40;
  if (a > CAP || b > CAP) return CAP;
  int64_t p = a * b;
  return p > CAP ? CAP : p;
}

}  // namespace

void tn::step_layouts(tn::Step& st) {
  const int n = st.n;
  st.y_off.assign(n, 0);
  int64_t off = 0;
  for (int k = 0; k < n; ++k) {
    const tn::SiteOp& o = st.site[k];
    st.y_off[k] = off;
    off += int64_t(o.a) * o.dhl * o.de * o.b * o.dhr;
  }
  st.y_total = off;
  // boundary sites after the step
  st.s_off.assign(n, 0);
  st.s_size.assign(n, 0);
  off = 0;
  for (int k = 0; k < n; ++k) {
    int64_t sz;
    if (st.kind == 0) {
      const tn::SiteOp& o = st.site[k];
      sz = int64_t(o.a) * o.dhl * o.de * o.b * o.dhr;
    } else if (st.kind == 1) {
      const int64_t left = (k == 0) ? 1 : st.r[k - 1];
      const int64_t right = (k == n - 1) ? 1 : st.r[k];
      sz = left * st.d[k] * right;
    } else {
      sz = 0;
    }
    st.s_off[k] = off;
    st.s_size[k] = sz;
    off += sz;
  }
  st.s_total = off;
  st.r_off.assign(n, 0);
  off = 0;
  if (st.kind == 1) {
    for (int k = 1; k <= n - 1; ++k) {
      st.r_off[k] = off;
      off += int64_t(st.D[k]) * st.D[k];
    }
  }
  st.r_total = off;
}

namespace {

void boundary_steps(const tn_graph* g, const tn_plan_opts* o, tn_plan_t* P,
                    const std::vector<std::vector<int>>& members, const std::vector<int>& path,
                    const std::vector<std::vector<int>>& inc);

void build(const tn_graph* g, const tn_plan_opts* o, tn_plan_t* P) {
  if (!g || !o) fail(TN_ERR_INVALID, "graph and opts must be non-NULL");
  const int nv = g->n_vertices, ne = g->n_edges;
  if (nv < 2) fail(TN_ERR_INVALID, "need at least 2 vertices");
  if (ne < 0) fail(TN_ERR_INVALID, "n_edges < 0");
  if (ne > 0 && (!g->edge_u || !g->edge_v || !g->edge_dim))
    fail(TN_ERR_INVALID, "edge arrays must be non-NULL");
  if (o->chi_max < 1) fail(TN_ERR_INVALID, "chi_max must be >= 1");
  if (o->ansatz != 0) fail(TN_ERR_UNSUPPORTED, "only the MPS ansatz (0) is implemented");
  for (int e = 0; e < ne; ++e) {
    const int u = g->edge_u[e], v = g->edge_v[e];
    if (u < 0 || u >= nv) fail(TN_ERR_INVALID, "edge endpoint out of range");
    if (v == -1) fail(TN_ERR_UNSUPPORTED, "open edges: the network must be closed");
    if (v < 0 || v >= nv) fail(TN_ERR_INVALID, "edge endpoint out of range");
    if (u == v) fail(TN_ERR_INVALID, "self loop");
    if (g->edge_dim[e] < 1) fail(TN_ERR_INVALID, "edge dim < 1");
  }
  // parts
  std::vector<int> part(nv);
  int nparts = 0;
  if (o->partition) {
    for (int v = 0; v < nv; ++v) {
      part[v] = o->partition[v];
      if (part[v] < 0 || part[v] >= nv) fail(TN_ERR_INVALID, "partition id out of range");
      nparts = std::max(nparts, part[v] + 1);
    }
  } else {
    if (o->env_size < 1) fail(TN_ERR_INVALID, "env_size must be >= 1 without a partition");
    for (int v = 0; v < nv; ++v) part[v] = v / o->env_size;
    nparts = (nv + o->env_size - 1) / o->env_size;
  }
  std::vector<std::vector<int>> members(nparts);
  for (int v = 0; v < nv; ++v) members[part[v]].push_back(v);
  for (int p = 0; p < nparts; ++p)
    if (members[p].empty()) fail(TN_ERR_INVALID, "empty part");
  if (nparts < 2) fail(TN_ERR_UNSUPPORTED, "need at least two parts");
  std::vector<int> path(nparts);
  if (o->path) {
    if (o->n_path != nparts) fail(TN_ERR_INVALID, "path must list every part once");
    std::vector<char> seen(nparts, 0);
    for (int i = 0; i < nparts; ++i) {
      const int p = o->path[i];
      if (p < 0 || p >= nparts || seen[p]) fail(TN_ERR_INVALID, "path is not a permutation");
      seen[p] = 1;
      path[i] = p;
    }
  } else {
    for (int i = 0; i < nparts; ++i) path[i] = i;
  }
  // incidence, tensor layouts (legs in ascending edge id)
  std::vector<std::vector<int>> inc(nv);
  for (int e = 0; e < ne; ++e) {
    inc[g->edge_u[e]].push_back(e);
    inc[g->edge_v[e]].push_back(e);
  }
  P->n_vertices = nv;
  P->n_edges = ne;
  P->chi = o->chi_max;
  P->site_off.assign(nv, 0);
  P->site_len.assign(nv, 0);
  int64_t off = 0;
  for (int v = 0; v < nv; ++v) {
    std::sort(inc[v].begin(), inc[v].end());
    int64_t len = 1;
    for (int e : inc[v]) len = cap_mul(len, g->edge_dim[e]);
    if (len >= (int64_t(1) << 31)) fail(TN_ERR_UNSUPPORTED, "site tensor too large");
    P->site_off[v] = off;
    P->site_len[v] = len;
    off += len;
  }
  P->site_elems = off;
  if (o->planner < 0 || o->planner > 1) fail(TN_ERR_INVALID, "planner must be 0 or 1");
  bool general = o->planner == 1;
  if (!general) {
    try {
      boundary_steps(g, o, P, members, path, inc);
      P->n_contractions = nparts - 1;
    } catch (const Fail& f) {
      if (f.st != TN_ERR_UNSUPPORTED) throw;
      general = true;
      P->steps.clear();
    }
  }
  if (general) {
    std::vector<std::vector<int>> parts;
    for (int s = 0; s < nparts; ++s) parts.push_back(members[path[s]]);
    tn::build_general_steps(g, o, parts, P);
  }
  tn::plan_info(P);
}

// Boundary absorption: every part a simple path whose i-th vertex absorbs the
// i-th open leg of the intermediate (the 2D lattice rows).
void boundary_steps(const tn_graph* g, const tn_plan_opts* o, tn_plan_t* P,
                    const std::vector<std::vector<int>>& members, const std::vector<int>& path,
                    const std::vector<std::vector<int>>& inc) {
  const int nv = g->n_vertices;
  const int nparts = int(members.size());
  auto other = [&](int e, int v) { return g->edge_u[e] == v ? g->edge_v[e] : g->edge_u[e]; };
  auto stride_of = [&](int v, int e) {
    int64_t s = 1;
    const auto& l = inc[v];
    for (int j = int(l.size()) - 1; j >= 0; --j) {
      if (l[j] == e) return s;
      s *= g->edge_dim[l[j]];
    }
    return int64_t(-1);
  };
  std::vector<char> absorbed(nv, 0);
  std::vector<int> legs;                          // open legs of the intermediate (edge ids)
  std::vector<int64_t> sa, sd, sb;                // boundary site shapes (a, d, b)
  for (int s = 0; s < nparts; ++s) {
    const std::vector<int>& mem = members[path[s]];
    const int m = int(mem.size());
    std::map<int, int> idx;
    for (int i = 0; i < m; ++i) idx[mem[i]] = i;
    std::vector<std::vector<int>> consumed(m), internal(m), fresh(m);
    for (int i = 0; i < m; ++i) {
      const int u = mem[i];
      for (int e : inc[u]) {
        const int w = other(e, u);
        if (absorbed[w]) consumed[i].push_back(e);
        else if (idx.count(w)) internal[i].push_back(e);
        else fresh[i].push_back(e);
      }
    }
    // order the part as a path
    std::vector<int> chain;
    if (s == 0) {
      int start = -1, nint = 0;
      for (int i = 0; i < m; ++i) {
        nint += int(internal[i].size());
        if (internal[i].size() > 2) fail(TN_ERR_UNSUPPORTED, "part is not a simple path");
        if (internal[i].size() <= 1 && start < 0) start = i;  // smallest-id endpoint (mem ascending)
      }
      if (nint != 2 * (m - 1) || start < 0) fail(TN_ERR_UNSUPPORTED, "part is not a simple path");
      std::vector<char> used(m, 0);
      int cur = start, prev_e = -1;
      while (cur >= 0) {
        chain.push_back(cur);
        used[cur] = 1;
        int nxt = -1;
        for (int e : internal[cur]) {
          if (e == prev_e) continue;
          const int j = idx[other(e, mem[cur])];
          if (!used[j]) { nxt = j; prev_e = e; break; }
        }
        cur = nxt;
      }
      if (int(chain.size()) != m) fail(TN_ERR_UNSUPPORTED, "part is not a connected path");
    } else {
      if (m != int(legs.size()))
        fail(TN_ERR_UNSUPPORTED, "every part must absorb all open legs, one per vertex");
      std::map<int, int> pos;
      for (int k = 0; k < int(legs.size()); ++k) pos[legs[k]] = k;
      chain.assign(m, -1);
      for (int i = 0; i < m; ++i) {
        if (consumed[i].size() != 1)
          fail(TN_ERR_UNSUPPORTED, "each part vertex must absorb exactly one open leg");
        const int k = pos.at(consumed[i][0]);
        chain[k] = i;
      }
    }
    // check path edges are exactly consecutive pairs, once each
    int nint = 0;
    for (int i = 0; i < m; ++i) nint += int(internal[i].size());
    if (nint != 2 * (m - 1)) fail(TN_ERR_UNSUPPORTED, "part is not a simple path");
    tn::Step st;
    st.n = m;
    st.kind = (s == 0) ? 0 : (s == nparts - 1 ? 2 : 1);
    st.site.resize(m);
    st.d.assign(m, 1);
    st.D.assign(m, 1);
    std::vector<int> new_legs;
    for (int k = 0; k < m; ++k) {
      const int i = chain[k];
      const int u = mem[i];
      tn::SiteOp op{};
      op.vertex = u;
      op.t_off = P->site_off[u];
      op.dp = op.dhl = op.dhr = op.de = 1;
      op.sp = op.shl = op.shr = op.se = 0;
      int hl = -1, hr = -1;
      for (int e : internal[i]) {
        const int j = idx[other(e, u)];
        if (k > 0 && j == chain[k - 1] && hl < 0) hl = e;
        else if (k + 1 < m && j == chain[k + 1] && hr < 0) hr = e;
        else fail(TN_ERR_UNSUPPORTED, "part edges must join consecutive path vertices once");
      }
      if (k > 0 && hl < 0) fail(TN_ERR_UNSUPPORTED, "part path is broken");
      if (hl >= 0) { op.dhl = g->edge_dim[hl]; op.shl = stride_of(u, hl); }
      if (hr >= 0) { op.dhr = g->edge_dim[hr]; op.shr = stride_of(u, hr); }
      if (s > 0) {
        const int e = consumed[i][0];
        op.dp = g->edge_dim[e];
        op.sp = stride_of(u, e);
        op.a = int32_t(sa[k]);
        op.b = int32_t(sb[k]);
        if (sd[k] != op.dp) fail(TN_ERR_INVALID, "boundary leg dim mismatch");
      } else {
        op.a = op.b = 1;
      }
      if (fresh[i].size() > 1)
        fail(TN_ERR_UNSUPPORTED, "a part vertex may emit at most one new open leg");
      if (fresh[i].size() == 1) {
        const int e = fresh[i][0];
        op.de = g->edge_dim[e];
        op.se = stride_of(u, e);
        new_legs.push_back(e);
      } else if (st.kind != 2) {
        fail(TN_ERR_UNSUPPORTED, "every vertex of a non-final part must emit one open leg");
      }
      st.site[k] = op;
      st.d[k] = op.de;
    }
    for (int k = 0; k < m; ++k) {
      const tn::SiteOp& op = st.site[k];
      const int64_t left = int64_t(op.a) * op.dhl, right = int64_t(op.b) * op.dhr;
      if (left >= (1 << 20) || right >= (1 << 20)) fail(TN_ERR_UNSUPPORTED, "bond too large");
      st.D[k] = int32_t(right);
      if (k > 0 && st.D[k - 1] != left) fail(TN_ERR_INVALID, "inconsistent bond dims");
    }
    if (st.kind == 1 && m < 3) fail(TN_ERR_UNSUPPORTED, "intermediates need >= 3 open legs");
    // ranks of the density-matrix pass
    if (st.kind == 1) {
      st.r.assign(m - 1, 0);
      st.r[0] = st.d[0];
      for (int k = 1; k <= m - 2; ++k) {
        int64_t beyond = 1;
        for (int j = k + 1; j < m; ++j) beyond = cap_mul(beyond, st.d[j]);
        int64_t r = std::min<int64_t>(o->chi_max, int64_t(st.r[k - 1]) * st.d[k]);
        r = std::min<int64_t>(r, st.D[k]);
        r = std::min<int64_t>(r, beyond);
        st.r[k] = int32_t(r);
      }
    }
    // boundary after the step
    sa.assign(m, 1); sd.assign(m, 1); sb.assign(m, 1);
    for (int k = 0; k < m; ++k) {
      const tn::SiteOp& op = st.site[k];
      sd[k] = st.d[k];
      if (st.kind == 0) {
        sa[k] = int64_t(op.a) * op.dhl;
        sb[k] = st.D[k];
      } else if (st.kind == 1) {
        sa[k] = (k == 0) ? 1 : st.r[k - 1];
        sb[k] = (k == m - 1) ? 1 : st.r[k];
      }
    }
    tn::step_layouts(st);
    P->steps.push_back(std::move(st));
    for (int u : mem) absorbed[u] = 1;
    legs = new_legs;
  }
}

}  // namespace

// Plan summary and flop counts (Sec. 2.2 cost model, 2 flops per multiply-add).
void tn::plan_info(tn_plan_t* P) {
  tn_plan_info& I = P->info;
  std::memset(&I, 0, sizeof(I));
  I.n_steps = P->n_contractions;
  I.n_exec_steps = int32_t(P->steps.size());
  I.general = (!P->steps.empty() && P->steps.back().general) ? 1 : 0;
  I.site_elems = P->site_elems;
  for (const tn::Step& st : P->steps) {
    I.max_legs = std::max(I.max_legs, st.n);
    for (int k = 0; k < st.n; ++k) I.max_bond = std::max(I.max_bond, st.D[k]);
    if (st.kind != 1) continue;
    I.n_dm_passes++;
    const int n = st.n;
    for (int k = n - 1; k >= 2; --k) {
      const double Dl = st.D[k - 1], dk = st.d[k], Dr = st.D[k];
      I.flops_env += 2.0 * Dl * dk * Dr * Dr + 2.0 * Dl * Dl * dk * Dr;
    }
    for (int k = 1; k <= n - 2; ++k) {
      const double rp = st.r[k - 1], Dl = st.D[k - 1], dk = st.d[k], Dr = st.D[k];
      const double A = rp * dk, r = st.r[k];
      I.flops_local += 2.0 * rp * Dl * dk * Dr;
      I.flops_density += 2.0 * A * Dr * Dr + 2.0 * A * A * Dr;
      I.flops_project += 2.0 * r * A * Dr;
      I.flops_eig += (4.0 / 3.0) * A * A * A + 4.0 * A * A * r;
      // factored form: Cholesky of R_v, K_v = M_v C_v, bidiagonal SVD of K_v
      I.flops_factor += Dr * Dr * Dr / 3.0;
      I.flops_kfactor += 2.0 * A * Dr * Dr;
      I.flops_svd += (A >= Dr ? 4.0 * A * Dr * Dr - (4.0 / 3.0) * Dr * Dr * Dr
                              : 4.0 * Dr * A * A - (4.0 / 3.0) * A * A * A) +
                     2.0 * A * A * r;
      I.max_eig_n = std::max(I.max_eig_n, int32_t(A));
      I.n_eig++;
    }
    I.flops_project += 2.0 * st.r[n - 2] * st.D[n - 2] * st.d[n - 1];
  }
}

extern "C" tn_status tn_plan(const tn_graph* graph, const tn_plan_opts* opts, tn_plan_t** out) {
  if (!out) {
    set_error("tn_plan: out is NULL");
    return TN_ERR_INVALID;
  }
  *out = nullptr;
  tn_plan_t* P = new (std::nothrow) tn_plan_t();
  if (!P) {
    set_error("tn_plan: host allocation failed");
    return TN_ERR_OOM;
  }
  try {
    build(graph, opts, P);
  } catch (const Fail& f) {
    delete P;
    set_error("tn_plan: " + f.msg);
    return f.st;
  } catch (const std::bad_alloc&) {
    delete P;
    set_error("tn_plan: host allocation failed");
    return TN_ERR_OOM;
  } catch (...) {
    delete P;
    set_error("tn_plan: unexpected error");
    return TN_ERR_INVALID;
  }
  *out = P;
  return TN_OK;
}

extern "C" tn_status tn_plan_destroy(tn_plan_t* plan) {
  delete plan;
  return TN_OK;
}

extern "C" tn_status tn_plan_query(const tn_plan_t* plan, tn_plan_info* info) {
  if (!plan || !info) {
    set_error("tn_plan_query: NULL argument");
    return TN_ERR_INVALID;
  }
  *info = plan->info;
  return TN_OK;
}

extern "C" tn_status tn_plan_step_query(const tn_plan_t* plan, int32_t step, tn_plan_step* info,
                                        int32_t* leaves, int32_t* d, int32_t* D, int32_t* r) {
  if (!plan || step < 0 || step >= int32_t(plan->steps.size())) {
    set_error("tn_plan_step_query: invalid argument");
    return TN_ERR_INVALID;
  }
  const tn::Step& st = plan->steps[step];
  if (info) {
    info->kind = st.kind;
    info->n = st.n;
    info->n_kt = st.n_kt;
    info->general = st.general ? 1 : 0;
  }
  for (int k = 0; k < st.n; ++k) {
    if (leaves) leaves[k] = (st.general && st.kind == 1) ? st.leaves[k] : -1;
    if (d) d[k] = st.d[k];
    if (D) D[k] = st.D[k];
    if (r && st.kind == 1 && k + 1 < st.n) r[k] = st.r[k];
  }
  return TN_OK;
}

extern "C" tn_status tn_plan_site_offset(const tn_plan_t* plan, int32_t vertex, int64_t* offset) {
  if (!plan || !offset || vertex < 0 || vertex >= plan->n_vertices) {
    set_error("tn_plan_site_offset: invalid argument");
    return TN_ERR_INVALID;
  }
  *offset = plan->site_off[vertex];
  return TN_OK;
}
