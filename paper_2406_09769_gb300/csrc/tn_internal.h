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

// General plans build the block of every chain position (its tensors
// contracted together, with a delta for every edge passing through) by a
// short program of gather-contractions: pairwise contractions of the tensors
// in a greedy order into scratch, then one final op that writes the block.
// Per op, code[code_off ..] holds the slot dims (ns), the output slots (nout,
// row-major digits, the first slowest; a slot listed twice is a delta) and
// the summed slots (nsum).  Ops of one level are independent.
struct GOpH {
  int32_t pos, level;            // chain position, launch level
  int32_t to_block;              // 1: writes the block Y_pos, 0: scratch
  int64_t dst_off;               // scratch offset (elements per instance)
  int64_t n_elems;               // output elements
  int32_t Dl, dkDr;              // block shape (to_block): rows, columns
  int32_t ns, nout, nsum, nt, t_first, code_off;
};
// An operand of an op: src 0 = graph vertex id (its packed site tensor times
// its inverse norm), src 1 = site id of the MPS the previous step wrote,
// src 2 = scratch at offset id.  code[leg_off ..]: (slot, stride) per leg.
struct GTensorH {
  int32_t src, id, nleg, leg_off;
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
  // general plans: blocks built by the gather kernel instead of SiteOp fusion
  bool general = false;
  std::vector<GOpH> gop;         // sorted by level
  std::vector<int32_t> level_start;  // ops of level j: [level_start[j], level_start[j+1])
  int64_t scratch_elems = 0;     // per instance
  std::vector<GTensorH> gten;
  std::vector<int32_t> gcode;
  std::vector<int32_t> leaves;   // graph edge of every leaf (DM passes)
  int32_t n_kt = 0;              // Kendall-Tau distance of the contraction
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
  int32_t n_contractions = 0;    // contractions on the path (parts - 1)
  tn_plan_info info{};
};

namespace tn {
// Thread-local last error for calls without a ctx.
void set_error(const std::string& msg);
const char* get_error();
bool plans_equivalent(const tn_plan_t* a, const tn_plan_t* b);
// Planner failure (caught by tn_plan and turned into its status).
struct PlanFail {
  tn_status st;
  std::string msg;
};
// General planner (any graph, any partition): appends the steps of the
// maximally unbalanced path over parts (vertex lists in path order) to P.
void build_general_steps(const tn_graph* g, const tn_plan_opts* o,
                         std::vector<std::vector<int>> parts, tn_plan_t* P);
// Shared by both planners: per-step buffer layouts and the plan's flop counts.
void step_layouts(Step& st);
void plan_info(tn_plan_t* P);
}  // namespace tn
