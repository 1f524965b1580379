// Internal structures shared by the planner (host C++) and the executor (CUDA).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "tn_dmtree.h"

namespace tn {

// Block fusion of one tree vertex ("contract T(v) first", Sec. 5.3):
//   Y[a, hl, e, b, hr] = sum_p S[a, p, b] * T_vertex[p, hl, hr, e] * inv_norm(vertex)
// S is the boundary site aligned with this vertex; the roles p (leg to an
// already absorbed part), hl/hr (path edges inside the part) and e (new open
// leg) are strided views of the vertex tensor (stride 0 and dim 1 if absent).
struct SiteOp {
  int32_t vertex;
  int64_t t_off;                 // vertex tensor offset in the packed site buffer
  int32_t dp, dhl, dhr, de;      // role dims
  int64_t sp, shl, shr, se;      // role strides (elements)
  int32_t a, b;                  // boundary site S: (a, dp, b)
};

struct Step {
  int32_t kind;                  // 0: first part (exact), 1: DM pass, 2: closing contraction
  int32_t n;                     // sites (open legs of the intermediate)
  std::vector<SiteOp> site;
  std::vector<int32_t> d;        // new leg dims d_k
  std::vector<int32_t> D;        // untruncated tree-edge dims D_k (D_{n-1} = 1)
  std::vector<int32_t> r;        // ranks after the pass r_0..r_{n-2} (DM pass only)
  // packed layouts (elements) of this step's per-instance buffers
  std::vector<int64_t> y_off;    // Y_k blocks
  int64_t y_total = 0;
  std::vector<int64_t> s_off;    // boundary sites after this step
  std::vector<int64_t> s_size;
  int64_t s_total = 0;
  std::vector<int64_t> r_off;    // memoised density matrices R_k (k = 1..n-2)
  int64_t r_total = 0;
};

}  // namespace tn

struct tn_plan {
  int32_t n_vertices = 0;
  int32_t n_edges = 0;
  int32_t chi = 0;
  std::vector<int64_t> site_off; // per vertex offset in the packed site buffer
  std::vector<int64_t> site_len;
  int64_t site_elems = 0;
  std::vector<tn::Step> steps;
  tn_plan_info info{};
};

namespace tn {
// Thread-local last error for calls without a ctx.
void set_error(const std::string& msg);
const char* get_error();
bool plans_equivalent(const tn_plan_t* a, const tn_plan_t* b);
}  // namespace tn
