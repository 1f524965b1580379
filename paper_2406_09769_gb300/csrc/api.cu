// C ABI entry points: device context, workspace, and the executor that runs a
// plan of Algorithm partitioned_contract on the GPU for a batch of instances.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "tn_internal.h"

namespace {

struct Fail {
  tn_status st;
  std::string msg;
};

[[noreturn]] void fail(tn_status st, const std::string& msg) { throw Fail{st, msg}; }

void ck(cudaError_t e, const char* what) {
  if (e != cudaSuccess) fail(TN_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Host-side allocation fault injection: TN_FAULT_ALLOC_AT=n makes the n-th
// device allocation of the process fail with TN_ERR_OOM (no CUDA call made).
long g_alloc_count = 0;
bool inject_alloc_failure() {
  static long at = [] {
    const char* s = std::getenv("TN_FAULT_ALLOC_AT");
    return s ? std::atol(s) : 0L;
  }();
  ++g_alloc_count;
  return at > 0 && g_alloc_count == at;
}

// A device buffer that only grows.
struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
  void* get(size_t bytes) {
    if (bytes <= cap) return p;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    if (inject_alloc_failure()) fail(TN_ERR_OOM, "device allocation failed (injected)");
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      fail(TN_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    }
    cap = bytes;
    return p;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
};

}  // namespace

struct tn_ctx {
  int device = 0;
  std::string err;
  cudaStream_t stream = nullptr;
  int last_batch = 0;
  bool pending = false;
  // workspace
  DevBuf arena, stage, tables, results;
  DevBuf gdesc;             // descriptor tables of grouped batches
  DevBuf gguard;            // range table of the grouped guard mode
  void* pinned = nullptr;
  size_t pinned_cap = 0;
  cudaEvent_t pinned_free = nullptr;
  // diagnostics: launch counts per kernel class, optional event timing
  bool prof = false;
  int64_t launches[TN_KC_COUNT] = {};
  struct Rec {
    int cls;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  bool tc_ready = false;  // tcgen05/TMA path configured on this device
  // learned per-edge rank allocation
  DevBuf model_buf;        // BF16 MLP parameters
  int chi_uniform = 0;
  bool have_model = false;
  DevBuf learn_buf;        // per-instance running budgets
  float* rec_feat = nullptr;
  double* rec_spec = nullptr;
  int* rec_chi = nullptr;
  double* rec_acc = nullptr;
  int64_t rec_cap = 0;     // edges (eigensolves) the record buffers hold per instance
  DevBuf train_buf;        // gradient and Adam moments
  DevBuf aux_buf;          // label tables, sample indices
  // the uniform-chi judge of learned ranks (learned_chi = 2)
  int hook_fixed_chi = 0;  // > 0: the rank hook keeps min(chi_uniform, r_v), no model
  double* hook_acc = nullptr;  // overrides rec_acc as the discarded-share accumulator
  DevBuf judge_buf;        // acc_l, acc_u, logz_u, status_u, used
  int* judged = nullptr;   // per instance: 1 = learned run kept (last judged batch)
  int judged_n = 0;
  // device pointers carved from `results`
  double* logz = nullptr;
  int* status = nullptr;
  double* logscale = nullptr;
  int* err_flag = nullptr;  // set by a kernel whose bounded wait expired
  int* poll_flag = nullptr; // a device flag that nothing sets (TN_OPT_WAIT_PROBE)
  // options (tn_ctx_set_option)
  int eig_rounds = 9;       // SVD multisection rounds after the grid round
  bool value_comp = true;   // compensated accumulation on the value path
  bool grouped = true;      // mixed batches of many general plans run grouped
  bool wait_probe = false;  // next batch: bounded wait on poll_flag in the GEMMs
  // result slot of each instance of the last batch (bucketed batches)
  std::vector<int> slot;
  bool slot_identity = true;
  // autotuned tensor-core tiles: {M, N, K, split, batch} -> {tile width, smem budget KB}
  std::map<std::array<int, 5>, std::array<int, 3>> tune;  // value: BN, budget KB, time (ns)
  bool tuning = false;
  // concurrent buckets: a pool of streams with fork / join events
  std::vector<cudaStream_t> pool;
  std::vector<cudaEvent_t> joins;
  cudaEvent_t fork = nullptr;
  cudaEvent_t gready = nullptr;  // grouped batches: tables and site norms done
};

namespace {

struct Ws {
  // per-instance strides (elements) and base pointers
  long long sS, sY, sR, sX, sM, sL, sP, sLam, sAmax, sInv, sScr;
  double *S0, *S1, *Y, *R, *X, *M, *G, *L, *P, *lam, *inv, *scr;
  unsigned long long* amax;
};

struct Dims {
  long long maxS = 1, maxY = 1, maxR = 1, maxX = 1, maxM = 1, maxL = 1, maxP = 1, maxLam = 1,
            maxScr = 1;
  int maxN = 1, maxD = 1;
};

Dims plan_dims(const tn_plan_t* P) {
  Dims d;
  for (const tn::Step& st : P->steps) {
    d.maxS = std::max<long long>(d.maxS, st.s_total);
    d.maxY = std::max<long long>(d.maxY, st.y_total);
    d.maxR = std::max<long long>(d.maxR, st.r_total);
    d.maxScr = std::max<long long>(d.maxScr, st.scratch_elems);
    d.maxN = std::max(d.maxN, st.n);
    for (int k = 0; k < st.n; ++k) {
      d.maxD = std::max(d.maxD, st.D[k]);
      const tn::SiteOp& o = st.site[k];
      d.maxX = std::max<long long>(d.maxX, (long long)o.a * o.dhl * o.de * o.b * o.dhr);
    }
    if (st.kind != 1) continue;
    for (int k = 1; k <= st.n - 2; ++k) {
      const long long A = (long long)st.r[k - 1] * st.d[k];
      d.maxM = std::max<long long>(d.maxM, A * st.D[k]);
      d.maxL = std::max<long long>(d.maxL, A * A);
      d.maxP = std::max<long long>(d.maxP, (long long)st.r[k] * st.D[k]);
      d.maxLam = std::max<long long>(d.maxLam, A);
    }
  }
  return d;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// bytes: if set, receives the workspace size; with dry = true nothing is
// allocated and the returned pointers are not valid.
Ws carve(tn_ctx* c, const Dims& d, int B, int nv, bool dry = false, size_t* bytes = nullptr,
         char* at = nullptr) {
  Ws w{};
  w.sS = d.maxS; w.sY = d.maxY; w.sR = d.maxR; w.sX = d.maxX; w.sM = d.maxM;
  w.sL = d.maxL; w.sP = d.maxP; w.sLam = d.maxLam; w.sAmax = d.maxN; w.sInv = nv;
  w.sScr = d.maxScr;
  const size_t dbl = sizeof(double);
  size_t off[16];
  size_t tot = 0;
  const long long sizes[] = {w.sS, w.sS, w.sY, w.sR, w.sX, w.sM, w.sM, w.sL, w.sP, w.sLam, w.sInv,
                             w.sScr};
  for (int i = 0; i < 12; ++i) {
    off[i] = tot;
    tot += align256(dbl * size_t(sizes[i]) * B);
  }
  off[12] = tot;
  tot += align256(sizeof(unsigned long long) * size_t(w.sAmax) * B);
  if (bytes) *bytes = tot;
  if (dry) return w;
  char* base = at ? at : static_cast<char*>(c->arena.get(tot));
  double** outs[] = {&w.S0, &w.S1, &w.Y, &w.R, &w.X, &w.M, &w.G, &w.L, &w.P, &w.lam, &w.inv,
                     &w.scr};
  for (int i = 0; i < 12; ++i) *outs[i] = reinterpret_cast<double*>(base + off[i]);
  w.amax = reinterpret_cast<unsigned long long*>(base + off[12]);
  return w;
}

void ensure_results(tn_ctx* c, int B) {
  char* base = static_cast<char*>(c->results.get(align256(sizeof(double) * B) * 2 +
                                                 align256(sizeof(int) * B) + 256));
  c->logz = reinterpret_cast<double*>(base);
  c->logscale = reinterpret_cast<double*>(base + align256(sizeof(double) * B));
  c->status = reinterpret_cast<int*>(base + 2 * align256(sizeof(double) * B));
  c->err_flag = reinterpret_cast<int*>(base + 2 * align256(sizeof(double) * B) +
                                       align256(sizeof(int) * B));
  c->poll_flag = c->err_flag + 1;
}

// Per-step buffer offsets (elements) of one executor.
struct Lay {
  std::vector<int64_t> y_off, s_off, r_off;
  int64_t y_total = 0, s_total = 0, r_total = 0;
};

Lay lay_fp64(const tn::Step& st) {
  Lay l;
  l.y_off = st.y_off;
  l.s_off = st.s_off;
  l.r_off = st.r_off;
  l.y_total = st.y_total;
  l.s_total = st.s_total;
  l.r_total = st.r_total;
  return l;
}

int64_t up4(int64_t x) { return (x + 3) & ~int64_t(3); }

// 16-byte aligned FP32 offsets (TMA needs 16-byte aligned bases and strides).
Lay lay_f32(const tn::Step& st) {
  Lay l;
  const int n = st.n;
  l.y_off.assign(n, 0);
  l.s_off.assign(n, 0);
  l.r_off.assign(n, 0);
  int64_t off = 0;
  for (int k = 0; k < n; ++k) {
    const tn::SiteOp& o = st.site[k];
    l.y_off[k] = off;
    off += up4(int64_t(o.a) * o.dhl * o.de * o.b * o.dhr);
  }
  l.y_total = off;
  off = 0;
  for (int k = 0; k < n; ++k) {
    l.s_off[k] = off;
    off += up4(st.s_size[k]);
  }
  l.s_total = off;
  off = 0;
  if (st.kind == 1)
    for (int k = 1; k <= n - 1; ++k) {
      l.r_off[k] = off;
      off += up4(int64_t(st.D[k]) * st.D[k]);
    }
  l.r_total = off;
  return l;
}

// Counts one launch of a kernel class and, when profiling, brackets it with
// CUDA events on the launching stream.
struct Scope {
  tn_ctx* c;
  int cls;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  Scope(tn_ctx* c_, int cls_, cudaStream_t s_) : c(c_), cls(cls_), s(s_) {
    if (c->prof && cudaEventCreate(&a) == cudaSuccess) cudaEventRecord(a, s);
  }
  ~Scope() {
    c->launches[cls]++;
    cudaEvent_t b = nullptr;
    if (a && cudaEventCreate(&b) == cudaSuccess) {
      cudaEventRecord(b, s);
      c->recs.push_back({cls, a, b});
    }
  }
};

void* pinned_get(tn_ctx* c, size_t bytes) {
  ck(cudaEventSynchronize(c->pinned_free), "cudaEventSynchronize");
  if (bytes > c->pinned_cap) {
    if (c->pinned) cudaFreeHost(c->pinned);
    c->pinned = nullptr;
    c->pinned_cap = 0;
    if (cudaMallocHost(&c->pinned, bytes) != cudaSuccess) {
      cudaGetLastError();
      fail(TN_ERR_OOM, "pinned host allocation failed");
    }
    c->pinned_cap = bytes;
  }
  return c->pinned;
}

// Device copies of the plan's per-step tables.
struct StepTables {
  tn::FuseSite* fuse;
  int64_t* y_off;
  int32_t* D;      // n + 1 entries (last = max D)
  int64_t* r_off;  // memoised density matrix R_k offsets (n entries)
  // general plans: the block programs (ops by level, operands, code, prefix)
  tn::GOp* gop;
  tn::GTen* gten;
  int32_t* gcode;
  int64_t* gpre;
};

size_t general_bytes(const tn::Step& st) {
  if (!st.general) return 0;
  return align256(sizeof(tn::GOp) * st.gop.size()) + align256(sizeof(tn::GTen) * st.gten.size()) +
         align256(sizeof(int32_t) * st.gcode.size()) +
         align256(sizeof(int64_t) * (st.gop.size() + 1));
}

// Device copies of one bucket's per-step tables: [tens ptrs B][site_off nv]
// [site_len nv] then per step fuse / y_off / D / r_off.
size_t tables_bytes(const tn_plan_t* P, int B) {
  const int nv = P->n_vertices;
  size_t tot = align256(sizeof(void*) * B) + 2 * align256(sizeof(int64_t) * nv);
  for (size_t s = 0; s < P->steps.size(); ++s) {
    const int n = P->steps[s].n;
    tot += align256(sizeof(tn::FuseSite) * n) + 2 * align256(sizeof(int64_t) * n) +
           align256(sizeof(int32_t) * (n + 1)) + general_bytes(P->steps[s]);
  }
  return tot;
}

// Lays out the tables at device address dbase; writes their host image at h
// when h is not NULL (h == NULL: the device copy is already in place).
std::vector<StepTables> fill_tables(const tn_plan_t* P, const std::vector<Lay>& lay,
                                    const double* const* tens_dev, int B, char* h, char* dbase,
                                    const double*** tens_table, int64_t** off_dev,
                                    int64_t** len_dev) {
  const int nv = P->n_vertices;
  size_t o = align256(sizeof(void*) * B);
  if (h) std::memcpy(h, tens_dev, sizeof(void*) * B);
  if (h) std::memcpy(h + o, P->site_off.data(), sizeof(int64_t) * nv);
  *off_dev = reinterpret_cast<int64_t*>(dbase + o);
  o += align256(sizeof(int64_t) * nv);
  if (h) std::memcpy(h + o, P->site_len.data(), sizeof(int64_t) * nv);
  *len_dev = reinterpret_cast<int64_t*>(dbase + o);
  o += align256(sizeof(int64_t) * nv);
  *tens_table = reinterpret_cast<const double**>(dbase);
  std::vector<StepTables> out(P->steps.size());
  for (size_t s = 0; s < P->steps.size(); ++s) {
    const tn::Step& stp = P->steps[s];
    const int n = stp.n;
    size_t q = o;
    out[s].fuse = reinterpret_cast<tn::FuseSite*>(dbase + q);
    if (h) {
      tn::FuseSite* fh = reinterpret_cast<tn::FuseSite*>(h + q);
      for (int k = 0; k < n; ++k) {
        const tn::SiteOp& op = stp.site[k];
        tn::FuseSite f{};
        f.vertex = op.vertex; f.a = op.a; f.dp = op.dp; f.b = op.b;
        f.dhl = op.dhl; f.dhr = op.dhr; f.de = op.de;
        f.t_off = op.t_off; f.sp = op.sp; f.shl = op.shl; f.shr = op.shr; f.se = op.se;
        f.y_off = (stp.kind == 0) ? lay[s].s_off[k] : lay[s].y_off[k];
        f.s_off = (s > 0 && !stp.general) ? lay[s - 1].s_off[k] : 0;
        fh[k] = f;
      }
    }
    q += align256(sizeof(tn::FuseSite) * n);
    if (h) std::memcpy(h + q, lay[s].y_off.data(), sizeof(int64_t) * n);
    out[s].y_off = reinterpret_cast<int64_t*>(dbase + q);
    q += align256(sizeof(int64_t) * n);
    if (h) {
      std::vector<int32_t> D(stp.D);
      int mx = 1;
      for (int x : D) mx = std::max(mx, x);
      D.push_back(mx);
      std::memcpy(h + q, D.data(), sizeof(int32_t) * (n + 1));
    }
    out[s].D = reinterpret_cast<int32_t*>(dbase + q);
    q += align256(sizeof(int32_t) * (n + 1));
    if (h) {
      std::vector<int64_t> ro(lay[s].r_off);
      ro.resize(n, 0);
      std::memcpy(h + q, ro.data(), sizeof(int64_t) * n);
    }
    out[s].r_off = reinterpret_cast<int64_t*>(dbase + q);
    q += align256(sizeof(int64_t) * n);
    out[s].gop = nullptr;
    out[s].gten = nullptr;
    out[s].gcode = nullptr;
    out[s].gpre = nullptr;
    if (stp.general) {
      const size_t nop = stp.gop.size(), nten = stp.gten.size(), ncode = stp.gcode.size();
      out[s].gop = reinterpret_cast<tn::GOp*>(dbase + q);
      if (h) {
        tn::GOp* gh = reinterpret_cast<tn::GOp*>(h + q);
        for (size_t i = 0; i < nop; ++i) {
          const tn::GOpH& x = stp.gop[i];
          tn::GOp g{};
          g.dst_off = x.to_block ? lay[s].y_off[x.pos] : x.dst_off;
          g.n_elems = x.n_elems;
          g.to_block = x.to_block; g.Dl = x.Dl; g.dkDr = x.dkDr;
          g.ns = x.ns; g.nout = x.nout; g.nsum = x.nsum; g.nt = x.nt;
          g.t_first = x.t_first; g.code_off = x.code_off;
          gh[i] = g;
        }
      }
      q += align256(sizeof(tn::GOp) * nop);
      out[s].gten = reinterpret_cast<tn::GTen*>(dbase + q);
      if (h) {
        tn::GTen* th = reinterpret_cast<tn::GTen*>(h + q);
        for (size_t i = 0; i < nten; ++i) {
          const tn::GTensorH& x = stp.gten[i];
          tn::GTen g{};
          g.src = x.src; g.nleg = x.nleg; g.leg_off = x.leg_off;
          if (x.src == 0) {
            g.base = P->site_off[x.id];
            g.vertex = x.id;
          } else if (x.src == 1) {
            g.base = lay[s - 1].s_off[x.id];
          } else {
            g.base = x.id;
          }
          th[i] = g;
        }
      }
      q += align256(sizeof(tn::GTen) * nten);
      out[s].gcode = reinterpret_cast<int32_t*>(dbase + q);
      if (h) std::memcpy(h + q, stp.gcode.data(), sizeof(int32_t) * ncode);
      q += align256(sizeof(int32_t) * ncode);
      out[s].gpre = reinterpret_cast<int64_t*>(dbase + q);
      if (h) {
        int64_t* ph = reinterpret_cast<int64_t*>(h + q);
        ph[0] = 0;
        for (size_t i = 0; i < nop; ++i) ph[i + 1] = ph[i] + stp.gop[i].n_elems;
      }
      q += align256(sizeof(int64_t) * (nop + 1));
    }
    o = q;
  }
  return out;
}

// One bucket of a batch: instances whose plans are structurally equal.
struct Bucket {
  const tn_plan_t* P = nullptr;
  std::vector<int> idx;                // instances of the batch, in order
  std::vector<const double*> sites;    // their site buffers
  std::vector<Lay> lay;
  size_t ws_bytes = 0, tab_off = 0, res_off = 0, ws_off = 0;
  char* ws_at = nullptr;  // workspace slice (concurrent buckets), NULL: the arena
  std::vector<StepTables> tabs;
  const double** tens_table = nullptr;
  int64_t *off_dev = nullptr, *len_dev = nullptr;
};

void gemm(tn_ctx* c, int cls, bool ta, bool tb, const double* A, long long sA, int lda,
          const double* Bm, long long sB, int ldb, double* C, long long sC, int ldc, int M, int N,
          int K, int batch, const unsigned long long* amax_in, long long s_in,
          unsigned long long* amax_out, long long s_out, cudaStream_t st) {
  Scope sc(c, cls, st);
  tn::GemmArgs g{};
  g.A = A; g.sA = sA; g.lda = lda;
  g.B = Bm; g.sB = sB; g.ldb = ldb;
  g.C = C; g.sC = sC; g.ldc = ldc;
  g.M = M; g.N = N; g.K = K; g.batch = batch;
  g.amax_in = amax_in; g.s_amax_in = s_in;
  g.amax_out = amax_out; g.s_amax_out = s_out;
  ck(tn::launch_dgemm(ta, tb, g, st), "dgemm launch");
}

// Per-pass context of the learned rank allocation and of spectrum recording.
struct PassCtx {
  int pass = 0, npass = 1;
  bool learned = false, record = false;
  int budget_total = 0;
  int* budget_rem = nullptr;
  long long* edge = nullptr;  // running eigensolve index of the contraction
};

int pass_budget(const tn::Step& st, int chi_u) {
  int b = 0;
  for (int k = 1; k <= st.n - 2; ++k) b += std::min(chi_u, st.r[k]);
  return b;
}

struct LearnState {
  bool learned = false, record = false;
  int* budget_rem = nullptr;
  long long edge = 0;
  int pass = 0, npass = 1;
};

LearnState learn_begin(tn_ctx* c, const tn_plan_t* P, int B, bool learned, cudaStream_t strm) {
  LearnState s;
  s.learned = learned || c->hook_fixed_chi > 0;
  s.record = c->hook_fixed_chi == 0 && (c->rec_feat || c->rec_spec || c->rec_chi || c->rec_acc);
  s.npass = std::max(1, int(P->info.n_dm_passes));
  if (s.learned || s.record) {
    s.budget_rem = static_cast<int*>(c->learn_buf.get(2 * sizeof(int) * size_t(B)));
    double* acc = c->hook_acc ? c->hook_acc : c->rec_acc;
    if (acc) ck(cudaMemsetAsync(acc, 0, sizeof(double) * size_t(B), strm), "memset acc");
  }
  return s;
}

PassCtx learn_pass(LearnState& s, tn_ctx* c, const tn::Step& st) {
  PassCtx pc;
  pc.pass = s.pass++;
  pc.npass = s.npass;
  pc.learned = s.learned;
  pc.record = s.record;
  pc.budget_total = c->chi_uniform > 0 ? pass_budget(st, c->chi_uniform) : 0;
  pc.budget_rem = s.budget_rem;
  pc.edge = &s.edge;
  return pc;
}

// After the eigensolve of vertex k: learned rank (mask U beyond chi) and/or records.
template <typename T>
void rank_hook(tn_ctx* c, const PassCtx* pc, const tn::Step& st, int k, int A, int rk,
               const double* lam, long long slam, T* U, long long sU, T* Ut, long long sUt, int B,
               cudaStream_t strm) {
  if (!pc || !(pc->learned || pc->record)) return;
  Scope sc(c, TN_KC_EIG, strm);
  tn::RankArgs g{};
  g.lam = lam; g.slam = slam; g.A = A; g.rk = rk; g.dk = st.d[k];
  g.v = k; g.nlegs = st.n; g.pass = pc->pass; g.npass = pc->npass;
  g.model = (pc->learned && c->hook_fixed_chi == 0) ? c->model_buf.p : nullptr;
  g.fixed_chi = c->hook_fixed_chi;
  g.budget_total = pc->budget_total;
  g.chi_uniform = c->chi_uniform;
  g.edges_after = st.n - 2 - k;
  g.reserve_after = 0;
  for (int u = k + 1; u <= st.n - 2; ++u) g.reserve_after += std::min(2, st.r[u]);
  g.first = (k == 1);
  g.budget_rem = pc->budget_rem;
  g.prev_chi = pc->budget_rem + B;
  g.acc = c->hook_acc ? c->hook_acc : c->rec_acc;
  const long long e = pc->edge ? (*pc->edge)++ : 0;
  if (pc->record && e < c->rec_cap) {
    g.rec_chi = c->rec_chi; g.rec_feat = c->rec_feat; g.rec_spec = c->rec_spec;
    g.rec_off = e * B;
  }
  ck(tn::launch_rank_select<T>(g, U, sU, Ut, sUt, B, strm), "rank select");
}

// One density_matrix_alg pass (Sec. 5) over the blocks in w.Y (layout of st),
// writing the tree TN as boundary sites into Snext (layout st.s_off).
void dm_pass(tn_ctx* c, const tn::Step& st, const Ws& w, double* Snext, int B, int precision,
             cudaStream_t strm, const PassCtx* pc = nullptr) {
  (void)precision;
  const bool want_lam = pc && (pc->learned || pc->record);
  const int n = st.n;
  const auto& D = st.D;
  const auto& d = st.d;
  // Memoised root-side density matrices, Eq. (dm_cache):
  //   R_{n-1} = [1];  R_{k-1} = sum_e Y_k(:, e, :) R_k Y_k(:, e, :)^T  (k = n-1 .. 2)
  // Each R_k is kept unnormalised; its running max-abs (amax[k]) scales the
  // GEMM that consumes it, which keeps every R within range.
  ck(cudaMemsetAsync(w.amax, 0, sizeof(unsigned long long) * w.sAmax * B, strm), "memset amax");
  Scope(c, TN_KC_ENV, strm),
  ck(tn::launch_fill_env_root(w.R + st.r_off[n - 1], w.sR, w.amax + (n - 1), w.sAmax, B, strm),
     "env root");
  for (int k = n - 1; k >= 2; --k) {
    const double* Yk = w.Y + st.y_off[k];
    const int Dl = D[k - 1], Dr = D[k], dk = d[k];
    // X = Y_k (Dl*dk x Dr) . R_k / max|R_k|
    gemm(c, TN_KC_ENV, false, false, Yk, w.sY, Dr, w.R + st.r_off[k], w.sR, Dr, w.X, w.sX, Dr, Dl * dk, Dr, Dr,
         B, w.amax + k, w.sAmax, nullptr, 0, strm);
    // R_{k-1} = X (Dl x dk*Dr) . Y_k(Dl x dk*Dr)^T
    gemm(c, TN_KC_ENV, false, true, w.X, w.sX, dk * Dr, Yk, w.sY, dk * Dr, w.R + st.r_off[k - 1], w.sR, Dl, Dl,
         Dl, dk * Dr, B, nullptr, 0, w.amax + (k - 1), w.sAmax, strm);
  }
  // Post-order over the MPS tree: vertices 1 .. n-2.
  for (int k = 1; k <= n - 2; ++k) {
    const int rp = st.r[k - 1], rk = st.r[k], dk = d[k], Dl = D[k - 1], Dr = D[k];
    const int A = rp * dk;
    const double* Pp = (k == 1) ? w.Y + st.y_off[0] : w.P;
    const long long sPp = (k == 1) ? w.sY : w.sP;
    // M_v = P_{v-1} . Y_v  -> (rp x dk*Dr) = (A x Dr)
    gemm(c, TN_KC_LOCAL, false, false, Pp, sPp, Dl, w.Y + st.y_off[k], w.sY, dk * Dr, w.M, w.sM, dk * Dr, rp,
         dk * Dr, Dl, B, nullptr, 0, nullptr, 0, strm);
    // L_v = M_v R_k M_v^T  (R_k scaled by 1/max|R_k|)
    gemm(c, TN_KC_DENSITY, false, false, w.M, w.sM, Dr, w.R + st.r_off[k], w.sR, Dr, w.G, w.sM, Dr, A, Dr, Dr, B,
         w.amax + k, w.sAmax, nullptr, 0, strm);
    gemm(c, TN_KC_DENSITY, false, true, w.G, w.sM, Dr, w.M, w.sM, Dr, w.L, w.sL, A, A, A, Dr, B, nullptr, 0, nullptr,
         0, strm);
    // U_v = leading_eigenvectors(L_v, r_k), written as boundary site k
    double* Uk = Snext + st.s_off[k];
    Scope(c, TN_KC_EIG, strm),
    ck(tn::launch_eigh_top<double>(w.L, w.sL, Uk, w.sS, nullptr, 0, w.lam, w.sLam, A, rk,
                                   want_lam ? A : 0, c->status, B, strm),
       "eigh launch");
    rank_hook<double>(c, pc, st, k, A, rk, w.lam, w.sLam, Uk, w.sS, nullptr, 0, B, strm);
    // P_v = U_v^T M_v  (rk x Dr)
    gemm(c, TN_KC_PROJECT, true, false, Uk, w.sS, rk, w.M, w.sM, Dr, w.P, w.sP, Dr, rk, Dr, A, B, nullptr, 0,
         nullptr, 0, strm);
  }
  // Root: M_r = P_{n-2} . Y_{n-1}, scaled to unit norm into the log-scale.
  Scope(c, TN_KC_ROOT, strm),
  ck(tn::launch_root(w.P, w.sP, w.Y + st.y_off[n - 1], w.sY, st.r[n - 2], D[n - 2], d[n - 1],
                     Snext + st.s_off[n - 1], Snext + st.s_off[0], d[0], w.sS, c->logscale,
                     c->status, B, strm),
     "root launch");
}

// Blocks of a general step: its gather-contraction programs, level by level.
template <typename TS, typename TY>
void gather_blocks(tn_ctx* c, const tn::Step& st, const StepTables& tab, const double** tens,
                   const double* inv, long long sInv, const TS* Scur, long long sS, double* scr,
                   long long sScr, TY* Y, long long sY, TY* Yt, int B, cudaStream_t strm) {
  std::vector<int64_t> pre(st.gop.size() + 1, 0);
  for (size_t i = 0; i < st.gop.size(); ++i) pre[i + 1] = pre[i] + st.gop[i].n_elems;
  for (size_t j = 0; j + 1 < st.level_start.size(); ++j) {
    const int a = st.level_start[j], b = st.level_start[j + 1];
    Scope(c, TN_KC_FUSE, strm),
    ck(tn::launch_gather<TS, TY>(tab.gop, tab.gten, tab.gcode, tab.gpre, a, b, pre[b] - pre[a],
                                 tens, inv, sInv, Scur, sS, scr, sScr, Y, sY, Yt, B, strm),
       "gather");
  }
}

// FP64 path of one bucket (tables in place, results at c->logz etc.).
void run_plan(tn_ctx* c, const Bucket& bk, int precision, bool learned, cudaStream_t strm) {
  const tn_plan_t* P = bk.P;
  const int B = int(bk.idx.size());
  const Dims dm = plan_dims(P);
  LearnState ls = learn_begin(c, P, B, learned, strm);
  const Ws w = carve(c, dm, B, P->n_vertices, false, nullptr, bk.ws_at);
  const double** tens_table = bk.tens_table;
  const int64_t* off_dev = bk.off_dev;
  const int64_t* len_dev = bk.len_dev;
  const std::vector<StepTables>& tabs = bk.tabs;
  Scope(c, TN_KC_NORM, strm),
  ck(tn::launch_site_norm(tens_table, off_dev, len_dev, P->n_vertices, B, w.inv, c->logscale,
                          c->status, strm),
     "site norm");
  double* Scur = w.S0;
  double* Snext = w.S1;
  for (size_t s = 0; s < P->steps.size(); ++s) {
    const tn::Step& st = P->steps[s];
    if (st.general) {
      gather_blocks<double, double>(c, st, tabs[s], tens_table, w.inv, w.sInv, Scur, w.sS, w.scr,
                                    w.sScr, w.Y, w.sY, nullptr, B, strm);
      if (st.kind == 1) {
        const PassCtx pc = learn_pass(ls, c, st);
        dm_pass(c, st, w, Snext, B, precision, strm, &pc);
        std::swap(Scur, Snext);
      } else {
        int maxD = 1;
        for (int k = 0; k < st.n; ++k) maxD = std::max(maxD, st.D[k]);
        Scope(c, TN_KC_CLOSE, strm),
        ck(tn::launch_close(w.Y, w.sY, tabs[s].y_off, tabs[s].D, st.n, maxD, c->logscale, c->logz,
                            c->status, B, strm),
           "close");
      }
      continue;
    }
    int maxe = 1;
    for (int k = 0; k < st.n; ++k) {
      const tn::SiteOp& o = st.site[k];
      maxe = std::max<int>(maxe, o.a * o.dhl * o.de * o.b * o.dhr);
    }
    if (st.kind == 0) {
      Scope(c, TN_KC_FUSE, strm),
      ck(tn::launch_fuse(tabs[s].fuse, st.n, maxe, tens_table, w.inv, P->n_vertices, nullptr, 0, 1,
                         Snext, w.sS, B, strm),
         "fuse");
      std::swap(Scur, Snext);
    } else if (st.kind == 1) {
      Scope(c, TN_KC_FUSE, strm),
      ck(tn::launch_fuse(tabs[s].fuse, st.n, maxe, tens_table, w.inv, P->n_vertices, Scur, w.sS, 0,
                         w.Y, w.sY, B, strm),
         "fuse");
      const PassCtx pc = learn_pass(ls, c, st);
      dm_pass(c, st, w, Snext, B, precision, strm, &pc);
      std::swap(Scur, Snext);
    } else {
      Scope(c, TN_KC_FUSE, strm),
      ck(tn::launch_fuse(tabs[s].fuse, st.n, maxe, tens_table, w.inv, P->n_vertices, Scur, w.sS, 0,
                         w.Y, w.sY, B, strm),
         "fuse");
      int maxD = 1;
      for (int k = 0; k < st.n; ++k) maxD = std::max(maxD, st.D[k]);
      Scope(c, TN_KC_CLOSE, strm),
      ck(tn::launch_close(w.Y, w.sY, tabs[s].y_off, tabs[s].D, st.n, maxD, c->logscale, c->logz,
                          c->status, B, strm),
         "close");
    }
  }
}

// ------------------------------------------------------ mixed precision path
// FP32 storage; density-matrix contractions (env, K_v or L_v) as TF32
// tensor-core products with FP32 accumulation (compensated 3-term split
// except in the fast mode); the value path (M_v, P_v) in FP32 FFMA, whose
// rounding has no common sign (the tensor-core accumulator's does); FP32
// eigensolver or SVD; root norm, log-scale and closing contraction in FP64.
struct WsF {
  long long sS, sY, sR, sX, sM, sL, sP, sUt, sLam, sAmax, sInv, sScr;
  float *S0, *S1, *Y, *Yt, *R, *X, *M, *Mt, *G, *L, *P, *Ut;
  double *lam, *inv, *scr;
  unsigned int* amax;
};

WsF carve_f32(tn_ctx* c, const tn_plan_t* P, const std::vector<Lay>& lay, int B,
              bool dry = false, size_t* bytes = nullptr, char* at = nullptr) {
  long long maxS = 4, maxY = 4, maxR = 4, maxX = 4, maxM = 4, maxL = 4, maxP = 4, maxUt = 4,
            maxLam = 1, maxScr = 1;
  int maxN = 1;
  for (size_t s = 0; s < P->steps.size(); ++s) {
    const tn::Step& st = P->steps[s];
    maxScr = std::max<long long>(maxScr, st.scratch_elems);
    maxS = std::max<long long>(maxS, lay[s].s_total);
    maxY = std::max<long long>(maxY, lay[s].y_total);
    maxR = std::max<long long>(maxR, lay[s].r_total);
    maxN = std::max(maxN, st.n);
    for (int k = 0; k < st.n; ++k) {
      const tn::SiteOp& o = st.site[k];
      maxX = std::max<long long>(maxX, up4((long long)o.a * o.dhl * o.de * o.b * o.dhr));
    }
    if (st.kind != 1) continue;
    for (int k = 1; k <= st.n - 2; ++k) {
      const long long A = (long long)st.r[k - 1] * st.d[k];
      maxM = std::max<long long>(maxM, up4(A * st.D[k]));
      maxL = std::max<long long>(maxL, up4(A * A));
      maxP = std::max<long long>(maxP, up4((long long)st.r[k] * st.D[k]));
      maxUt = std::max<long long>(maxUt, up4((long long)st.r[k] * A));
      maxLam = std::max<long long>(maxLam, A);
    }
  }
  WsF w{};
  w.sS = maxS; w.sY = maxY; w.sR = maxR; w.sX = maxX; w.sM = maxM; w.sL = maxL; w.sP = maxP;
  w.sUt = maxUt; w.sLam = maxLam; w.sAmax = maxN; w.sInv = P->n_vertices; w.sScr = maxScr;
  const long long fsz[] = {w.sS, w.sS, w.sY, w.sY, w.sR, w.sX, w.sM, w.sM, w.sM, w.sL, w.sP, w.sUt};
  float** fout[] = {&w.S0, &w.S1, &w.Y, &w.Yt, &w.R, &w.X, &w.M, &w.Mt, &w.G, &w.L, &w.P, &w.Ut};
  size_t off[16], tot = 0;
  for (int i = 0; i < 12; ++i) {
    off[i] = tot;
    tot += align256(sizeof(float) * size_t(fsz[i]) * B);
  }
  off[12] = tot;
  tot += align256(sizeof(double) * size_t(w.sLam) * B);
  off[13] = tot;
  tot += align256(sizeof(double) * size_t(w.sInv) * B);
  off[14] = tot;
  tot += align256(sizeof(double) * size_t(w.sScr) * B);
  off[15] = tot;
  tot += align256(sizeof(unsigned int) * size_t(w.sAmax) * B);
  if (bytes) *bytes = tot;
  if (dry) return w;
  char* base = at ? at : static_cast<char*>(c->arena.get(tot));
  for (int i = 0; i < 12; ++i) *fout[i] = reinterpret_cast<float*>(base + off[i]);
  w.lam = reinterpret_cast<double*>(base + off[12]);
  w.inv = reinterpret_cast<double*>(base + off[13]);
  w.scr = reinterpret_cast<double*>(base + off[14]);
  w.amax = reinterpret_cast<unsigned int*>(base + off[15]);
  return w;
}

// C_i = alpha_i A_i B_i^T on the tensor cores when TMA can address the operands
// (16-byte aligned bases and leading dimensions), else the SIMT fallback.
void tgemm(tn_ctx* c, int cls, const float* A, long long sA, int lda, const float* Bm,
           long long sB, int ldb, float* C, long long sC, int ldc, float* Ct, long long sCt,
           int ldct, int ct_cols, int M, int N, int K, int batch, const unsigned int* amax_in,
           long long s_in, unsigned int* amax_out, long long s_out, int split, cudaStream_t st) {
  Scope sc(c, cls, st);
  tn::TcGemmArgs g{};
  g.A = A; g.sA = sA; g.lda = lda;
  g.B = Bm; g.sB = sB; g.ldb = ldb;
  g.C = C; g.sC = sC; g.ldc = ldc;
  g.Ct = Ct; g.sCt = sCt; g.ldct = ldct; g.ct_cols = ct_cols > 0 ? ct_cols : N;
  g.M = M; g.N = N; g.K = K; g.batch = batch;
  g.amax_in = amax_in; g.s_amax_in = s_in;
  g.amax_out = amax_out; g.s_amax_out = s_out;
  g.split = split;
  g.err = c->err_flag;
  g.poll = c->wait_probe ? c->poll_flag : nullptr;
  const bool aligned = (lda % 4 == 0) && (ldb % 4 == 0) && (sA % 4 == 0) && (sB % 4 == 0) &&
                       (reinterpret_cast<uintptr_t>(A) % 16 == 0) &&
                       (reinterpret_cast<uintptr_t>(Bm) % 16 == 0);
  if (split == 2) {
    // value path: FP32 FFMA, rounding to nearest at every step
    ck(tn::launch_sgemm_ffma(g, c->value_comp, st), "ffma gemm launch");
    return;
  }
  if (aligned && c->tc_ready) {
    const std::array<int, 5> key{M, N, K, split, batch};
    if (c->tuning) {
      // time every candidate tile width and shared-memory budget once on the
      // real operands (all compute the same values: BN only partitions N and
      // the K order is fixed) and keep the fastest; the last run's output
      // stands
      std::vector<std::array<int, 2>> cand;
      const int nr = std::min(256, ((N + 15) / 16) * 16);
      for (int bn : {64, 128, 256}) {
        if (bn > std::max(64, nr)) continue;
        const int b = std::min(bn, nr);
        for (int kb : {70, 104, 200}) cand.push_back({b, kb});
      }
      cudaEvent_t e0, e1;
      ck(cudaEventCreate(&e0), "cudaEventCreate");
      ck(cudaEventCreate(&e1), "cudaEventCreate");
      std::array<int, 3> best{0, 0, 0};
      float best_ms = 1e30f;
      for (const auto& cd : cand) {
        g.bn = cd[0];
        g.budget_kb = cd[1];
        ck(cudaEventRecord(e0, st), "cudaEventRecord");
        ck(tn::launch_tc_gemm(g, st), "tcgen05 gemm launch");
        ck(cudaEventRecord(e1, st), "cudaEventRecord");
        ck(cudaEventSynchronize(e1), "cudaEventSynchronize");
        float ms = 0.f;
        ck(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
        if (ms < best_ms) {
          best_ms = ms;
          best = {cd[0], cd[1], int(ms * 1e6f)};
        }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      c->tune[key] = best;
      g.bn = best[0];
      g.budget_kb = best[1];
    } else {
      const auto it = c->tune.find(key);
      if (it != c->tune.end()) {
        g.bn = it->second[0];
        g.budget_kb = it->second[1];
      }
    }
    ck(tn::launch_tc_gemm(g, st), "tcgen05 gemm launch");
  } else {
    ck(tn::launch_sgemm_nt(g, st), "sgemm launch");
  }
}

// sub_split: compensated products also on the density-matrix side (env, L_v).
// factored: R_k = C_k C_k^T and the leading left singular vectors of
// K_v = M_v C_k instead of forming L_v (tab: this step's device tables).
void dm_pass_tc(tn_ctx* c, const tn::Step& st, const Lay& l, const WsF& w, float* Snext, int B,
                int sub_split, bool factored, const StepTables* tab, cudaStream_t strm,
                const PassCtx* pc = nullptr) {
  const bool want_lam = pc && (pc->learned || pc->record);
  const int n = st.n;
  const auto& D = st.D;
  const auto& d = st.d;
  ck(cudaMemsetAsync(w.amax, 0, sizeof(unsigned int) * w.sAmax * B, strm), "memset amax");
  Scope(c, TN_KC_ENV, strm),
  ck(tn::launch_fill_env_root_f32(w.R + l.r_off[n - 1], w.sR, w.amax + (n - 1), w.sAmax, B, strm),
     "env root");
  // Memoised root-side density matrices, Eq. (dm_cache).
  // B = R_k enters as its own transpose: R_k is symmetric.
  for (int k = n - 1; k >= 2; --k) {
    const float* Yk = w.Y + l.y_off[k];
    const int Dl = D[k - 1], Dr = D[k], dk = d[k];
    tgemm(c, TN_KC_ENV, Yk, w.sY, Dr, w.R + l.r_off[k], w.sR, Dr, w.X, w.sX, Dr, nullptr, 0, 0, 0,
          Dl * dk, Dr, Dr, B, w.amax + k, w.sAmax, nullptr, 0, sub_split, strm);
    tgemm(c, TN_KC_ENV, w.X, w.sX, dk * Dr, Yk, w.sY, dk * Dr, w.R + l.r_off[k - 1], w.sR, Dl,
          nullptr, 0, 0, 0, Dl, Dl, dk * Dr, B, nullptr, 0, w.amax + (k - 1), w.sAmax, sub_split,
          strm);
  }
  if (factored && n >= 3) {
    // R_k = C_k C_k^T for every vertex of the pass, C_k^T in place of R_k
    int maxD = 1;
    for (int k = 1; k <= n - 2; ++k) maxD = std::max(maxD, D[k]);
    Scope(c, TN_KC_FACTOR, strm),
    ck(tn::launch_chol_env(w.R, w.sR, tab->r_off, tab->D, maxD, w.amax, w.sAmax, 1, n - 2, B,
                           strm),
       "cholesky launch");
  }
  for (int k = 1; k <= n - 2; ++k) {
    const int rp = st.r[k - 1], rk = st.r[k], dk = d[k], Dl = D[k - 1], Dr = D[k];
    const int A = rp * dk;
    const float* Pp = (k == 1) ? w.Y + l.y_off[0] : w.P;
    const long long sPp = (k == 1) ? w.sY : w.sP;
    // M_v = P_{v-1} Y_v (value path, FP32 FFMA); also M_v^T for the projector.
    tgemm(c, TN_KC_LOCAL, Pp, sPp, Dl, w.Yt + l.y_off[k], w.sY, Dl, w.M, w.sM, dk * Dr, w.Mt,
          w.sM, A, Dr, rp, dk * Dr, Dl, B, nullptr, 0, nullptr, 0, 2, strm);
    float* Uk = Snext + l.s_off[k];
    if (factored) {
      // K_v = M_v C_k (C_k^T stored row-major: the K-major second operand)
      tgemm(c, TN_KC_DENSITY, w.M, w.sM, Dr, w.R + l.r_off[k], w.sR, Dr, w.G, w.sM, Dr, nullptr,
            0, 0, 0, A, Dr, Dr, B, nullptr, 0, nullptr, 0, 1, strm);
      // U_v = leading left singular vectors of K_v = leading eigenvectors of L_v
      Scope(c, TN_KC_EIG, strm),
      ck(tn::launch_svd_left(w.G, w.sM, A, Dr, Uk, w.sS, w.Ut, w.sUt, w.lam, w.sLam, rk,
                             want_lam ? A : 0, c->status, B, strm, c->eig_rounds),
         "svd launch");
    } else {
      // L_v = M_v R_k M_v^T
      tgemm(c, TN_KC_DENSITY, w.M, w.sM, Dr, w.R + l.r_off[k], w.sR, Dr, w.G, w.sM, Dr, nullptr,
            0, 0, 0, A, Dr, Dr, B, w.amax + k, w.sAmax, nullptr, 0, sub_split, strm);
      tgemm(c, TN_KC_DENSITY, w.G, w.sM, Dr, w.M, w.sM, Dr, w.L, w.sL, A, nullptr, 0, 0, 0, A, A,
            Dr, B, nullptr, 0, nullptr, 0, sub_split, strm);
      Scope(c, TN_KC_EIG, strm),
      ck(tn::launch_eigh_top<float>(w.L, w.sL, Uk, w.sS, w.Ut, w.sUt, w.lam, w.sLam, A, rk,
                                    want_lam ? A : 0, c->status, B, strm),
         "eigh launch");
    }
    rank_hook<float>(c, pc, st, k, A, rk, w.lam, w.sLam, Uk, w.sS, w.Ut, w.sUt, B, strm);
    // P_v = U_v^T M_v (value path, FP32 FFMA)
    tgemm(c, TN_KC_PROJECT, w.Ut, w.sUt, A, w.Mt, w.sM, A, w.P, w.sP, Dr, nullptr, 0, 0, 0, rk,
          Dr, A, B, nullptr, 0, nullptr, 0, 2, strm);
  }
  Scope(c, TN_KC_ROOT, strm),
  ck(tn::launch_root_f32(w.P, w.sP, D[n - 2], w.Y + l.y_off[n - 1], w.sY, st.r[n - 2], D[n - 2],
                         d[n - 1], Snext + l.s_off[n - 1], Snext + l.s_off[0], d[0], w.sS,
                         c->logscale, c->status, B, strm),
     "root launch");
}

// The factored form fits a pass when every vertex has dim A_v <= 128, tree
// edge <= 128 and rank <= 64 (the register-resident Cholesky and SVD);
// TN_PREC_TF32 runs the other passes in the compensated Gram form.
bool factored_fits(const tn::Step& st) {
  for (int k = 1; k <= st.n - 2; ++k)
    if (!tn::svd_left_supported(st.r[k - 1] * st.d[k], st.D[k], st.r[k])) return false;
  return true;
}

// Mixed path of one bucket (tables in place, results at c->logz etc.).
void run_plan_tc(tn_ctx* c, const Bucket& bk, int sub_split, bool factored, bool learned,
                 cudaStream_t strm) {
  const tn_plan_t* P = bk.P;
  const int B = int(bk.idx.size());
  const std::vector<Lay>& lay = bk.lay;
  const WsF w = carve_f32(c, P, lay, B, false, nullptr, bk.ws_at);
  LearnState ls = learn_begin(c, P, B, learned, strm);
  const double** tens_table = bk.tens_table;
  const int64_t* off_dev = bk.off_dev;
  const int64_t* len_dev = bk.len_dev;
  const std::vector<StepTables>& tabs = bk.tabs;
  Scope(c, TN_KC_NORM, strm),
  ck(tn::launch_site_norm(tens_table, off_dev, len_dev, P->n_vertices, B, w.inv, c->logscale,
                          c->status, strm),
     "site norm");
  float* Scur = w.S0;
  float* Snext = w.S1;
  for (size_t s = 0; s < P->steps.size(); ++s) {
    const tn::Step& st = P->steps[s];
    if (st.general) {
      gather_blocks<float, float>(c, st, tabs[s], tens_table, w.inv, w.sInv, Scur, w.sS, w.scr,
                                  w.sScr, w.Y, w.sY, st.kind == 1 ? w.Yt : nullptr, B, strm);
      if (st.kind == 1) {
        const PassCtx pc = learn_pass(ls, c, st);
        dm_pass_tc(c, st, lay[s], w, Snext, B, sub_split, factored && factored_fits(st),
                   &tabs[s], strm, &pc);
        std::swap(Scur, Snext);
      } else {
        int maxD = 1;
        for (int k = 0; k < st.n; ++k) maxD = std::max(maxD, st.D[k]);
        Scope(c, TN_KC_CLOSE, strm),
        ck(tn::launch_close_f32(w.Y, w.sY, tabs[s].y_off, tabs[s].D, st.n, maxD, c->logscale,
                                c->logz, c->status, B, strm),
           "close");
      }
      continue;
    }
    int maxe = 1, maxdl = 1, maxj = 1, maxt = 1, maxa = 1, maxb = 1, other = 0;
    for (int k = 0; k < st.n; ++k) {
      const tn::SiteOp& o = st.site[k];
      maxe = std::max<int>(maxe, o.a * o.dhl * o.de * o.b * o.dhr);
      maxdl = std::max<int>(maxdl, o.a * o.dhl);
      maxj = std::max<int>(maxj, o.de * o.b * o.dhr);
      maxt = std::max<int>(maxt, o.dp * o.dhl * o.dhr * o.de);
      maxa = std::max<int>(maxa, o.a);
      maxb = std::max<int>(maxb, o.b);
      if (o.dp != 2 || o.dhl != 2 || o.dhr != 2 || o.de != 2 || lay[s].y_off[k] % 2 != 0) ++other;
    }
    const int bond2 = (other <= 2) ? 1 : 0;  // square-lattice rows: only the end sites differ
    if (st.kind == 0) {
      Scope(c, TN_KC_FUSE, strm),
      ck(tn::launch_fuse_f32(tabs[s].fuse, st.n, maxe, maxdl, maxj, maxt, maxa, maxb, bond2,
                             tens_table, w.inv,
                             P->n_vertices, nullptr, 0, 1, Snext, w.sS, nullptr, nullptr, B, strm),
         "fuse");
      std::swap(Scur, Snext);
    } else if (st.kind == 1) {
      Scope(c, TN_KC_FUSE, strm),
      ck(tn::launch_fuse_f32(tabs[s].fuse, st.n, maxe, maxdl, maxj, maxt, maxa, maxb, bond2,
                             tens_table, w.inv,
                             P->n_vertices, Scur, w.sS, 0, w.Y, w.sY, w.Yt, tabs[s].y_off, B,
                             strm),
         "fuse");
      const PassCtx pc = learn_pass(ls, c, st);
      dm_pass_tc(c, st, lay[s], w, Snext, B, sub_split, factored && factored_fits(st),
                   &tabs[s], strm, &pc);
      std::swap(Scur, Snext);
    } else {
      Scope(c, TN_KC_FUSE, strm),
      ck(tn::launch_fuse_f32(tabs[s].fuse, st.n, maxe, maxdl, maxj, maxt, maxa, maxb, bond2,
                             tens_table, w.inv,
                             P->n_vertices, Scur, w.sS, 0, w.Y, w.sY, nullptr, nullptr, B, strm),
         "fuse");
      int maxD = 1;
      for (int k = 0; k < st.n; ++k) maxD = std::max(maxD, st.D[k]);
      Scope(c, TN_KC_CLOSE, strm),
      ck(tn::launch_close_f32(w.Y, w.sY, tabs[s].y_off, tabs[s].D, st.n, maxD, c->logscale,
                              c->logz, c->status, B, strm),
         "close");
    }
  }
}

// ------------------------------------------------------ grouped mixed path
// A batch of general plans (random graphs: one bucket per instance) as one
// launch sequence.  Every bucket's path is a list of operations (block
// gathers level by level, environment GEMMs, Cholesky factors, per tree
// vertex the local block, density, eigenvectors and projection, the root,
// the closing contraction), each at a position (global step, pass section,
// tree vertex); the lists are merged so that the operations at the same
// position share one launch over the problems of all buckets that have one,
// each problem with its own pointers and shape (descriptor tables built on
// the host once per batch).  Contractions run in FP32 FFMA (value path with
// Kahan accumulation as on the bucketed path); eigenvectors by the factored
// SVD where the pass fits it, else the Gram form.
struct GLaunch {
  int kind;            // 0 gather, 1 env root, 2 gemm, 3 gemm (value path), 4 chol,
                       // 5 svd, 6 eigh, 7 root, 8 close
  int cls;             // kernel class (TN_KC_*) of the launch
  size_t off;          // byte offset of the descriptors in the table
  int count;
  int64_t p0, p1, p2;  // launch extents (max elements / max M, N / max m, n, r);
                       // close: bucket, step
  int grp = 0;         // bucket group (stream) of the launch
};

struct GBuild {
  std::vector<char> bytes;
  std::vector<GLaunch> launches;
};

// One operation of one bucket: its problems' descriptors and extents.
struct GOp1 {
  int kind, cls;
  int64_t p0, p1, p2;
  size_t esz;         // bytes per descriptor
  std::vector<char> d;
  std::array<int, 4> key;  // position in the path: step, section, index, sub-step
};

template <class D>
void push_op(std::vector<GOp1>& ops, std::array<int, 4> key, int kind, int cls,
             const std::vector<D>& ds, int64_t p0, int64_t p1 = 0, int64_t p2 = 0) {
  if (ds.empty()) return;
  GOp1 o{kind, cls, p0, p1, p2, sizeof(D), {}, key};
  o.d.resize(sizeof(D) * ds.size());
  std::memcpy(o.d.data(), ds.data(), o.d.size());
  ops.push_back(std::move(o));
}

bool grouped_eligible(const std::vector<Bucket>& bks) {
  for (const Bucket& bk : bks)
    for (const tn::Step& st : bk.P->steps) {
      if (!st.general) return false;
      if (st.kind == 1)
        for (int k = 1; k <= st.n - 2; ++k)
          if (st.r[k - 1] * st.d[k] > 128 || st.r[k] > 64) return false;
    }
  return true;
}

// The operation list of bucket b (see above); res_* are the batch's result
// arrays (bucket b's instances at b.res_off ..).
std::vector<GOp1> bucket_ops(const std::vector<Bucket>& bks, size_t b, const WsF& w,
                             bool factored, double* res_logscale, int* res_status,
                             const tn::GuardTab* guard) {
  const Bucket& bk = bks[b];
  const int B = int(bk.idx.size());
  std::vector<GOp1> ops;
  int cur = 0;  // which of S0 / S1 holds the current MPS
  auto S_of = [&](int which) { return which ? w.S1 : w.S0; };
  for (size_t s = 0; s < bk.P->steps.size(); ++s) {
    const tn::Step& st = bk.P->steps[s];
    const Lay& l = bk.lay[s];
    const StepTables& t = bk.tabs[s];
    // blocks: the gather programs, level by level
    for (size_t j = 0; j + 1 < st.level_start.size(); ++j) {
      const int a = st.level_start[j], e = st.level_start[j + 1];
      int64_t ne = 0;
      for (int q = a; q < e; ++q) ne += st.gop[q].n_elems;
      if (std::getenv("TN_GROUPED_CHECK")) {
        // every element an op of this level reads or writes lies in its buffer
        const int32_t* code = st.gcode.data();
        for (int q = a; q < e; ++q) {
          const tn::GOpH& op = st.gop[q];
          if (op.to_block ? l.y_off[op.pos] + op.n_elems > w.sY : op.dst_off + op.n_elems > w.sScr)
            fail(TN_ERR_INVALID, "grouped check: gather output out of range");
          for (int u = 0; u < op.nt; ++u) {
            const tn::GTensorH& g = st.gten[op.t_first + u];
            int64_t ext = 1;
            for (int v = 0; v < g.nleg; ++v)
              ext += int64_t(code[op.code_off + code[g.leg_off + 2 * v]] - 1) *
                     code[g.leg_off + 2 * v + 1];
            int64_t base, lim;
            if (g.src == 0) { base = bk.P->site_off[g.id]; lim = bk.P->site_elems; }
            else if (g.src == 1) { base = bk.lay[s - 1].s_off[g.id]; lim = w.sS; }
            else { base = g.id; lim = w.sScr; }
            if (base + ext > lim) fail(TN_ERR_INVALID, "grouped check: gather operand out of range");
          }
        }
      }
      std::vector<tn::GatherDesc> ds;
      for (int i = 0; i < B; ++i) {
        tn::GatherDesc d{};
        d.ops = t.gop; d.ten = t.gten; d.code = t.gcode; d.pre = t.gpre;
        d.raw = bk.sites[i];
        d.inv = w.inv + i * w.sInv;
        d.S = S_of(cur) + i * w.sS;
        d.scr = w.scr + i * w.sScr;
        d.Y = w.Y + i * w.sY;
        d.Yt = st.kind == 1 ? w.Yt + i * w.sY : nullptr;
        d.a = a; d.b = e;
        d.guard = guard;
        ds.push_back(d);
      }
      push_op(ops, {int(s), 0, int(j), 0}, 0, TN_KC_FUSE, ds, ne);
    }
    if (st.kind == 2) {  // the closing contraction
      GOp1 o{8, TN_KC_CLOSE, int64_t(b), int64_t(s), 0, 0, {}, {int(s), 1, 0, 0}};
      ops.push_back(std::move(o));
      continue;
    }
    if (st.kind != 1) continue;
    const int n = st.n;
    // start of the pass: R_{n-1} = [1], amax
    {
      std::vector<tn::EnvRootDesc> ds;
      for (int i = 0; i < B; ++i)
        ds.push_back({w.R + i * w.sR + l.r_off[n - 1], w.amax + i * w.sAmax, n, 0, guard});
      push_op(ops, {int(s), 2, 0, 0}, 1, TN_KC_ENV, ds, 0);
    }
    // memoised environments, tree vertex k = n - 1 .. 2
    for (int k = n - 1; k >= 2; --k) {
      const int Dl = st.D[k - 1], Dr = st.D[k], dk = st.d[k];
      std::vector<tn::GemmDesc> dx, dr;
      for (int i = 0; i < B; ++i) {
        const float* Yk = w.Y + i * w.sY + l.y_off[k];
        float* X = w.X + i * w.sX;
        tn::GemmDesc x{};
        x.A = Yk; x.lda = Dr; x.B = w.R + i * w.sR + l.r_off[k]; x.ldb = Dr;
        x.C = X; x.ldc = Dr; x.M = Dl * dk; x.N = Dr; x.K = Dr; x.ct_cols = Dr;
        x.amax_in = w.amax + i * w.sAmax + k;
        x.guard = guard;
        dx.push_back(x);
        tn::GemmDesc y{};
        y.A = X; y.lda = dk * Dr; y.B = Yk; y.ldb = dk * Dr;
        y.C = w.R + i * w.sR + l.r_off[k - 1]; y.ldc = Dl; y.M = Dl; y.N = Dl; y.K = dk * Dr;
        y.ct_cols = Dl; y.amax_out = w.amax + i * w.sAmax + (k - 1);
        y.guard = guard;
        dr.push_back(y);
      }
      push_op(ops, {int(s), 3, n - 1 - k, 0}, 2, TN_KC_ENV, dx, int64_t(Dl) * dk, Dr);
      push_op(ops, {int(s), 3, n - 1 - k, 1}, 2, TN_KC_ENV, dr, Dl, Dl);
    }
    const bool fact = factored && factored_fits(st);
    if (fact) {
      std::vector<tn::CholDesc> ds;
      for (int i = 0; i < B; ++i)
        for (int k = 1; k <= n - 2; ++k)
          ds.push_back({w.R + i * w.sR + l.r_off[k], w.amax + i * w.sAmax + k, st.D[k], 0, guard});
      push_op(ops, {int(s), 4, 0, 0}, 4, TN_KC_FACTOR, ds, 0);
    }
    // post-order over tree vertices k = 1 .. n - 2
    float* Snext = S_of(1 - cur);
    for (int k = 1; k <= n - 2; ++k) {
      const int rp = st.r[k - 1], rk = st.r[k], dk = st.d[k], Dl = st.D[k - 1], Dr = st.D[k];
      const int A = rp * dk;
      std::vector<tn::GemmDesc> dm_, dk_, dl_, dp_;
      std::vector<tn::SvdDesc> dsv;
      std::vector<tn::EighDesc> deg;
      for (int i = 0; i < B; ++i) {
        const float* Pp = (k == 1) ? w.Y + i * w.sY + l.y_off[0] : w.P + i * w.sP;
        float* M = w.M + i * w.sM;
        float* Mt = w.Mt + i * w.sM;
        float* G = w.G + i * w.sM;
        float* Ut = w.Ut + i * w.sUt;
        float* Uk = Snext + i * w.sS + l.s_off[k];
        tn::GemmDesc g{};
        g.A = Pp; g.lda = Dl; g.B = w.Yt + i * w.sY + l.y_off[k]; g.ldb = Dl;
        g.C = M; g.ldc = dk * Dr; g.Ct = Mt; g.ldct = A; g.ct_cols = Dr;
        g.M = rp; g.N = dk * Dr; g.K = Dl;
        g.guard = guard;
        dm_.push_back(g);
        tn::GemmDesc q{};
        q.A = M; q.lda = Dr; q.B = w.R + i * w.sR + l.r_off[k]; q.ldb = Dr;
        q.C = G; q.ldc = Dr; q.M = A; q.N = Dr; q.K = Dr; q.ct_cols = Dr;
        if (!fact) q.amax_in = w.amax + i * w.sAmax + k;  // G = M R_k / amax
        q.guard = guard;
        dk_.push_back(q);
        if (fact) {
          dsv.push_back({G, Uk, Ut, w.lam + i * w.sLam, res_status + bk.res_off + i, A, Dr, rk, 0,
                         guard});
        } else {
          float* L = w.L + i * w.sL;
          tn::GemmDesc h{};
          h.A = G; h.lda = Dr; h.B = M; h.ldb = Dr; h.C = L; h.ldc = A;
          h.M = A; h.N = A; h.K = Dr; h.ct_cols = A;
          h.guard = guard;
          dl_.push_back(h);
          deg.push_back({L, Uk, Ut, w.lam + i * w.sLam, res_status + bk.res_off + i, A, rk, 0, 0,
                         guard});
        }
        tn::GemmDesc pq{};
        pq.A = Ut; pq.lda = A; pq.B = Mt; pq.ldb = A; pq.C = w.P + i * w.sP; pq.ldc = Dr;
        pq.M = rk; pq.N = Dr; pq.K = A; pq.ct_cols = Dr;
        pq.guard = guard;
        dp_.push_back(pq);
      }
      push_op(ops, {int(s), 5, k, 0}, 3, TN_KC_LOCAL, dm_, rp, int64_t(dk) * Dr);
      push_op(ops, {int(s), 5, k, 1}, 2, TN_KC_DENSITY, dk_, A, Dr);
      push_op(ops, {int(s), 5, k, 2}, 2, TN_KC_DENSITY, dl_, A, A);
      push_op(ops, {int(s), 5, k, 3}, 5, TN_KC_EIG, dsv, A, Dr, rk);
      push_op(ops, {int(s), 5, k, 4}, 6, TN_KC_EIG, deg, A, rk);
      push_op(ops, {int(s), 5, k, 5}, 3, TN_KC_PROJECT, dp_, rk, Dr);
    }
    // root M_r = P_{n-2} Y_{n-1}, unit norm into the log-scale
    {
      std::vector<tn::RootDesc> ds;
      for (int i = 0; i < B; ++i) {
        tn::RootDesc d{};
        d.P = w.P + i * w.sP; d.Y = w.Y + i * w.sY + l.y_off[n - 1];
        d.S_root = Snext + i * w.sS + l.s_off[n - 1]; d.S_first = Snext + i * w.sS + l.s_off[0];
        d.logscale = res_logscale + bk.res_off + i;
        d.status = res_status + bk.res_off + i;
        d.ldp = st.D[n - 2]; d.r = st.r[n - 2]; d.D = st.D[n - 2]; d.d = st.d[n - 1];
        d.d0 = st.d[0];
        d.guard = guard;
        ds.push_back(d);
      }
      push_op(ops, {int(s), 6, 0, 0}, 7, TN_KC_ROOT, ds, int64_t(st.r[n - 2]) * st.d[n - 1]);
    }
    cur = 1 - cur;
  }
  return ops;
}

// Merges the buckets' operation lists into one launch list: the buckets
// advance in lockstep through global step s, pass section and tree vertex,
// and the operations at the same position share a launch.  (A list schedule
// led by the bucket with the most estimated work left merged fewer
// operations per launch and ran ~15% slower on the random-graph batch.)
// Closing contractions run alone: their launch takes one bucket's tables.
void merge_grouped(const std::vector<std::vector<GOp1>>& per, GBuild& gb) {
  const size_t nb = per.size();
  std::vector<size_t> h(nb, 0);
  while (true) {
    int lead = -1;
    for (size_t b = 0; b < nb; ++b)
      if (h[b] < per[b].size() &&
          (lead < 0 || per[b][h[b]].key < per[size_t(lead)][h[size_t(lead)]].key))
        lead = int(b);
    if (lead < 0) break;
    const GOp1& o = per[size_t(lead)][h[size_t(lead)]];
    if (o.kind == 8) {
      gb.launches.push_back({8, o.cls, 0, 1, o.p0, o.p1, 0});
      ++h[size_t(lead)];
      continue;
    }
    GLaunch L{o.kind, o.cls, (gb.bytes.size() + 255) & ~size_t(255), 0, 0, 0, 0};
    gb.bytes.resize(L.off);
    for (size_t b = 0; b < nb; ++b) {
      if (h[b] >= per[b].size()) continue;
      const GOp1& x = per[b][h[b]];
      if (x.kind != o.kind || x.key != o.key) continue;
      gb.bytes.insert(gb.bytes.end(), x.d.begin(), x.d.end());
      L.count += int(x.d.size() / x.esz);
      L.p0 = std::max(L.p0, x.p0);
      L.p1 = std::max(L.p1, x.p1);
      L.p2 = std::max(L.p2, x.p2);
      ++h[b];
    }
    gb.launches.push_back(L);
  }
}

// Splits the buckets into at most n_groups groups, each run as its own
// lockstep sequence on a stream of its own: buckets sorted by a cost proxy (per
// tree vertex of every pass, 0.2 + (min(A_v, D_v) / 128)^1.5, the eigenvector
// problem's size), then groups of 1, 1, 2, 4, 8, ... buckets from the most
// expensive down, the last group taking the rest.  The batch lasts as long as
// its slowest group, and a group's lockstep sequence is at least its most
// expensive member's path, stretched by every position where another member
// has more vertices or larger matrices: the few most expensive instances get
// groups of their own, the many cheap ones share.
std::vector<std::vector<size_t>> group_buckets(const std::vector<Bucket>& bks, size_t n_groups) {
  std::vector<std::pair<double, size_t>> cost;
  for (size_t b = 0; b < bks.size(); ++b) {
    double w = 0.0;
    for (const tn::Step& st : bks[b].P->steps)
      if (st.kind == 1)
        for (int k = 1; k <= st.n - 2; ++k) {
          const double p = std::min(st.r[k - 1] * st.d[k], st.D[k]);
          w += 0.2 + std::pow(p / 128.0, 1.5);
        }
    cost.push_back({w, b});
  }
  std::stable_sort(cost.begin(), cost.end(),
                   [](const std::pair<double, size_t>& a, const std::pair<double, size_t>& b) {
                     return a.first > b.first;
                   });
  std::vector<std::vector<size_t>> groups;
  size_t i = 0, size = 1;
  while (i < cost.size()) {
    const bool last = groups.size() + 1 >= std::max<size_t>(1, n_groups);
    const size_t take = last ? cost.size() - i : std::min(size, cost.size() - i);
    groups.emplace_back();
    for (size_t j = 0; j < take; ++j) groups.back().push_back(cost[i + j].second);
    i += take;
    if (groups.size() >= 2) size *= 2;
  }
  return groups;
}

// Builds the launch list of a grouped batch (see above): every group's
// lockstep list, the groups' launches interleaved round robin (so that the
// host issues all streams' work evenly).
void build_grouped(const std::vector<Bucket>& bks, const std::vector<WsF>& ws,
                   const std::vector<std::vector<size_t>>& groups, bool factored,
                   double* res_logscale, int* res_status, GBuild& gb,
                   const tn::GuardTab* guard = nullptr) {
  std::vector<GBuild> per_group(groups.size());
  for (size_t g = 0; g < groups.size(); ++g) {
    std::vector<std::vector<GOp1>> per;
    for (size_t b : groups[g])
      per.push_back(bucket_ops(bks, b, ws[b], factored, res_logscale, res_status, guard));
    merge_grouped(per, per_group[g]);
  }
  std::vector<size_t> base(groups.size(), 0), next(groups.size(), 0);
  for (size_t g = 0; g < groups.size(); ++g) {
    base[g] = (gb.bytes.size() + 255) & ~size_t(255);
    gb.bytes.resize(base[g]);
    gb.bytes.insert(gb.bytes.end(), per_group[g].bytes.begin(), per_group[g].bytes.end());
  }
  for (bool more = true; more;) {
    more = false;
    for (size_t g = 0; g < groups.size(); ++g) {
      if (next[g] >= per_group[g].launches.size()) continue;
      GLaunch L = per_group[g].launches[next[g]++];
      if (L.kind != 8) L.off += base[g];
      L.grp = int(g);
      gb.launches.push_back(L);
      more = true;
    }
  }
}

// Host-side range check of a grouped launch list (TN_GROUPED_CHECK=1): every
// workspace operand of every descriptor must lie inside its bucket's
// workspace slice; the first violation is reported and nothing launches.
void check_grouped(const std::vector<Bucket>& bks, const GBuild& gb) {
  std::vector<std::pair<uintptr_t, uintptr_t>> sl;
  for (const Bucket& bk : bks) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(bk.ws_at);
    sl.push_back({a, a + bk.ws_bytes});
  }
  std::sort(sl.begin(), sl.end());
  auto inside = [&](const void* p, long long elems, size_t esz) {
    if (!p || elems <= 0) return true;
    const uintptr_t a = reinterpret_cast<uintptr_t>(p), e = a + uintptr_t(elems) * esz;
    auto it = std::upper_bound(sl.begin(), sl.end(), std::make_pair(a, ~uintptr_t(0)));
    if (it == sl.begin()) return false;
    --it;
    return a >= it->first && e <= it->second;
  };
  auto bad = [&](const char* what, size_t li, int q) {
    fail(TN_ERR_INVALID, std::string("grouped check: ") + what + " out of its slice, launch " +
                             std::to_string(li) + " problem " + std::to_string(q));
  };
  for (size_t li = 0; li < gb.launches.size(); ++li) {
    const GLaunch& g = gb.launches[li];
    const char* d = gb.bytes.data() + g.off;
    for (int q = 0; q < g.count && g.kind != 8; ++q) {
      if (g.kind == 2 || g.kind == 3) {
        const tn::GemmDesc x = reinterpret_cast<const tn::GemmDesc*>(d)[q];
        if (x.M > g.p0 || x.N > g.p1) bad("gemm extent", li, q);
        if (!inside(x.A, (long long)(x.M - 1) * x.lda + x.K, 4)) bad("gemm A", li, q);
        if (!inside(x.B, (long long)(x.N - 1) * x.ldb + x.K, 4)) bad("gemm B", li, q);
        if (!inside(x.C, (long long)(x.M - 1) * x.ldc + x.N, 4)) bad("gemm C", li, q);
        if (x.Ct && !inside(x.Ct, (long long)(x.ct_cols - 1) * x.ldct + (long long)x.M *
                                      (x.N / x.ct_cols), 4))
          bad("gemm Ct", li, q);
        if (x.lda < x.K || x.ldb < x.K || x.ldc < x.N) bad("gemm leading dim", li, q);
      } else if (g.kind == 5) {
        const tn::SvdDesc x = reinterpret_cast<const tn::SvdDesc*>(d)[q];
        if (x.m > g.p0 || x.n > g.p1 || x.r > g.p2 || x.r > x.m || x.r > x.n) bad("svd extent", li, q);
        if (!inside(x.K, (long long)x.m * x.n, 4)) bad("svd K", li, q);
        if (!inside(x.U, (long long)x.m * x.r, 4)) bad("svd U", li, q);
        if (!inside(x.Ut, (long long)x.m * x.r, 4)) bad("svd Ut", li, q);
      } else if (g.kind == 6) {
        const tn::EighDesc x = reinterpret_cast<const tn::EighDesc*>(d)[q];
        if (x.n > g.p0 || x.r > g.p1) bad("eigh extent", li, q);
        if (!inside(x.L, (long long)x.n * x.n, 4)) bad("eigh L", li, q);
        if (!inside(x.U, (long long)x.n * x.r, 4)) bad("eigh U", li, q);
        if (!inside(x.Ut, (long long)x.n * x.r, 4)) bad("eigh Ut", li, q);
      } else if (g.kind == 4) {
        const tn::CholDesc x = reinterpret_cast<const tn::CholDesc*>(d)[q];
        if (!inside(x.R, (long long)x.n * x.n, 4) || x.n > 128) bad("chol R", li, q);
        if (!inside(x.amax, 1, 4)) bad("chol amax", li, q);
      } else if (g.kind == 7) {
        const tn::RootDesc x = reinterpret_cast<const tn::RootDesc*>(d)[q];
        if ((long long)x.r * x.d > g.p0) bad("root extent", li, q);
        if (!inside(x.P, (long long)(x.r - 1) * x.ldp + x.D, 4)) bad("root P", li, q);
        if (!inside(x.Y, (long long)x.D * x.d, 4)) bad("root Y", li, q);
        if (!inside(x.S_root, (long long)x.r * x.d, 4)) bad("root S", li, q);
        if (!inside(x.S_first, (long long)x.d0 * x.d0, 4)) bad("root S_first", li, q);
      } else if (g.kind == 1) {
        const tn::EnvRootDesc x = reinterpret_cast<const tn::EnvRootDesc*>(d)[q];
        if (!inside(x.R, 1, 4) || !inside(x.amax, x.n, 4)) bad("env root", li, q);
      } else if (g.kind == 0) {
        const tn::GatherDesc x = reinterpret_cast<const tn::GatherDesc*>(d)[q];
        if (!inside(x.Y, 1, 4) || !inside(x.scr, 1, 8) || !inside(x.inv, 1, 8)) bad("gather", li, q);
      }
    }
  }
}

void run_grouped_tc(tn_ctx* c, const std::vector<Bucket>& bks, bool factored, bool upload,
                    double* res_logz, double* res_logscale, int* res_status, cudaStream_t strm) {
  std::vector<WsF> ws;
  for (const Bucket& bk : bks)
    ws.push_back(carve_f32(c, bk.P, bk.lay, int(bk.idx.size()), false, nullptr, bk.ws_at));
  for (size_t b = 0; b < bks.size(); ++b) {
    const Bucket& bk = bks[b];
    Scope(c, TN_KC_NORM, strm),
    ck(tn::launch_site_norm(bk.tens_table, bk.off_dev, bk.len_dev, bk.P->n_vertices,
                            int(bk.idx.size()), ws[b].inv, res_logscale + bk.res_off,
                            res_status + bk.res_off, strm),
       "site norm");
  }
  // guard mode (TN_GROUPED_GUARD=1, a diagnostic): every kernel checks its
  // global accesses against the batch's allocations, the host synchronises
  // after each launch and reports the first access outside them
  const char* genv = std::getenv("TN_GROUPED_GUARD");
  const bool guard_mode = genv && genv[0] == '1';
  tn::GuardTab* gdev = nullptr;
  unsigned long long* grec = nullptr;
  struct Rg {
    unsigned long long lo, hi;
    std::string what;
  };
  std::vector<Rg> labelled;
  if (guard_mode) {
    auto addr = [](const void* q) { return (unsigned long long)reinterpret_cast<uintptr_t>(q); };
    for (size_t b = 0; b < bks.size(); ++b) {
      const Bucket& bk = bks[b];
      labelled.push_back({addr(bk.ws_at), addr(bk.ws_at) + bk.ws_bytes,
                          "workspace of bucket " + std::to_string(b)});
      for (size_t i = 0; i < bk.sites.size(); ++i)
        labelled.push_back({addr(bk.sites[i]),
                            addr(bk.sites[i]) + sizeof(double) * size_t(bk.P->site_elems),
                            "sites of bucket " + std::to_string(b) + " instance " +
                                std::to_string(i)});
    }
    labelled.push_back({addr(c->tables.p), addr(c->tables.p) + c->tables.cap, "tables"});
    labelled.push_back({addr(c->results.p), addr(c->results.p) + c->results.cap, "results"});
    std::vector<std::pair<unsigned long long, unsigned long long>> rg;
    for (const Rg& r : labelled) rg.push_back({r.lo, r.hi});
    std::sort(rg.begin(), rg.end());
    std::vector<std::pair<unsigned long long, unsigned long long>> mg;
    for (const auto& r : rg) {
      if (!mg.empty() && r.first <= mg.back().second) mg.back().second = std::max(mg.back().second, r.second);
      else mg.push_back(r);
    }
    const int nr = int(mg.size());
    const size_t head = 256, recb = 4 * sizeof(unsigned long long);
    const size_t gbytes = head + recb + 2 * sizeof(unsigned long long) * size_t(nr);
    char* gbase = static_cast<char*>(c->gguard.get(gbytes));
    std::vector<char> img(gbytes, 0);
    tn::GuardTab t{};
    t.rec = reinterpret_cast<unsigned long long*>(gbase + head);
    t.lo = reinterpret_cast<unsigned long long*>(gbase + head + recb);
    t.hi = t.lo + nr;
    t.n = nr;
    std::memcpy(img.data(), &t, sizeof(t));
    for (int i = 0; i < nr; ++i) {
      std::memcpy(img.data() + head + recb + sizeof(unsigned long long) * i, &mg[i].first, 8);
      std::memcpy(img.data() + head + recb + sizeof(unsigned long long) * (nr + i), &mg[i].second, 8);
    }
    ck(cudaStreamSynchronize(strm), "guard: sync");
    ck(cudaMemcpy(gbase, img.data(), gbytes, cudaMemcpyHostToDevice), "guard: upload ranges");
    gdev = reinterpret_cast<tn::GuardTab*>(gbase);
    grec = t.rec;
  }
  // bucket groups on the pool streams (one group on strm in guard mode)
  const bool multi = !guard_mode && !c->pool.empty() && bks.size() >= 8;
  const std::vector<std::vector<size_t>> groups =
      group_buckets(bks, multi ? c->pool.size() : 1);
  std::vector<cudaStream_t> gs;
  for (size_t g = 0; g < groups.size(); ++g) gs.push_back(multi ? c->pool[g] : strm);
  GBuild gb;
  build_grouped(bks, ws, groups, factored, res_logscale, res_status, gb, gdev);
  if (const char* e = std::getenv("TN_GROUPED_CHECK"))
    if (e[0] == '1') {
      check_grouped(bks, gb);
      std::string st;
      for (int kd = 0; kd <= 8; ++kd) {
        long long n = 0, mc = 0, m0 = 0, m1 = 0, m2 = 0;
        for (const GLaunch& g : gb.launches)
          if (g.kind == kd) {
            ++n; mc = std::max<long long>(mc, g.count); m0 = std::max<long long>(m0, g.p0);
            m1 = std::max<long long>(m1, g.p1); m2 = std::max<long long>(m2, g.p2);
          }
        st += " k" + std::to_string(kd) + ":" + std::to_string(n) + "/" + std::to_string(mc) +
              "/" + std::to_string(m0) + "," + std::to_string(m1) + "," + std::to_string(m2);
      }
      fail(TN_ERR_INVALID, "grouped check passed (" + std::to_string(gb.launches.size()) +
                               " launches, " + std::to_string(gb.bytes.size()) + " bytes;" +
                               st + "); nothing launched");
    }
  char* dbase = static_cast<char*>(c->gdesc.get(std::max<size_t>(gb.bytes.size(), 256)));
  if (upload && !gb.bytes.empty())
    ck(cudaMemcpyAsync(dbase, gb.bytes.data(), gb.bytes.size(), cudaMemcpyHostToDevice, strm),
       "upload grouped tables");
  if (multi) {  // every group stream starts after the tables and the site norms
    if (!c->gready) ck(cudaEventCreateWithFlags(&c->gready, cudaEventDisableTiming),
                       "cudaEventCreate");
    ck(cudaEventRecord(c->gready, strm), "cudaEventRecord");
    for (cudaStream_t q : gs) ck(cudaStreamWaitEvent(q, c->gready, 0), "cudaStreamWaitEvent");
  }
  if (guard_mode && !gb.bytes.empty()) {
    std::vector<char> back(gb.bytes.size());
    ck(cudaStreamSynchronize(strm), "guard: sync");
    ck(cudaMemcpy(back.data(), dbase, back.size(), cudaMemcpyDeviceToHost), "guard: read back");
    if (std::memcmp(back.data(), gb.bytes.data(), back.size()) != 0)
      fail(TN_ERR_INVALID, "guard: device descriptor tables differ from the host image");
  }
  if (guard_mode && !gb.bytes.empty()) {
    // the descriptor tables lie outside every allowed range
    const unsigned long long d0 = (unsigned long long)reinterpret_cast<uintptr_t>(dbase);
    const unsigned long long d1 = d0 + gb.bytes.size();
    for (const Rg& r : labelled)
      if (r.lo < d1 && d0 < r.hi)
        fail(TN_ERR_INVALID, "guard: descriptor tables overlap " + r.what);
  }
  auto where = [&](unsigned long long a) {
    const Rg* best = nullptr;
    for (const Rg& r : labelled)
      if (r.lo <= a && (!best || r.lo > best->lo)) best = &r;
    if (!best) return std::string("below every allocation");
    return best->what + " +" + std::to_string(a - best->lo) + " (size " +
           std::to_string(best->hi - best->lo) + ")";
  };
  auto launch_bytes = [&](const GLaunch& g) -> size_t {
    switch (g.kind) {
      case 0: return sizeof(tn::GatherDesc) * size_t(g.count);
      case 1: return sizeof(tn::EnvRootDesc) * size_t(g.count);
      case 2: case 3: return sizeof(tn::GemmDesc) * size_t(g.count);
      case 4: return sizeof(tn::CholDesc) * size_t(g.count);
      case 5: return sizeof(tn::SvdDesc) * size_t(g.count);
      case 6: return sizeof(tn::EighDesc) * size_t(g.count);
      case 7: return sizeof(tn::RootDesc) * size_t(g.count);
      default: return 0;
    }
  };
  for (size_t li = 0; li < gb.launches.size(); ++li) {
    const GLaunch& g = gb.launches[li];
    char* d = dbase + g.off;
    cudaStream_t ls = gs[size_t(g.grp)];
    if (guard_mode && launch_bytes(g)) {
      // this launch's descriptors are still as uploaded
      std::vector<char> back(launch_bytes(g));
      ck(cudaMemcpy(back.data(), d, back.size(), cudaMemcpyDeviceToHost), "guard: read back");
      for (size_t q = 0; q < back.size(); ++q)
        if (back[q] != gb.bytes[g.off + q])
          fail(TN_ERR_INVALID, "guard: descriptors of launch " + std::to_string(li) + " kind " +
                                   std::to_string(g.kind) + " changed on the device at byte " +
                                   std::to_string(q) + " of " + std::to_string(back.size()) +
                                   " (table offset " + std::to_string(g.off) + ")");
    }
    switch (g.kind) {
      case 0:
        Scope(c, g.cls, ls),
        ck(tn::launch_gather_grouped(reinterpret_cast<tn::GatherDesc*>(d), g.count, g.p0, guard_mode,
                                     ls),
           "grouped gather");
        break;
      case 1:
        Scope(c, g.cls, ls),
        ck(tn::launch_env_root_grouped(reinterpret_cast<tn::EnvRootDesc*>(d), g.count, ls),
           "grouped env root");
        break;
      case 2:
      case 3:
        Scope(c, g.cls, ls),
        ck(tn::launch_gemm_grouped(reinterpret_cast<tn::GemmDesc*>(d), g.count, int(g.p0),
                                   int(g.p1), g.kind == 3 && c->value_comp, guard_mode, ls),
           "grouped gemm");
        break;
      case 4:
        Scope(c, g.cls, ls),
        ck(tn::launch_chol_grouped(reinterpret_cast<tn::CholDesc*>(d), g.count, guard_mode, ls),
           "grouped cholesky");
        break;
      case 5:
        Scope(c, g.cls, ls),
        ck(tn::launch_svd_left_grouped(reinterpret_cast<tn::SvdDesc*>(d), g.count, int(g.p0),
                                       int(g.p1), int(g.p2), guard_mode, ls, c->eig_rounds),
           "grouped svd");
        break;
      case 6:
        Scope(c, g.cls, ls),
        ck(tn::launch_eigh_grouped(reinterpret_cast<tn::EighDesc*>(d), g.count, int(g.p0),
                                   int(g.p1), guard_mode, ls),
           "grouped eigh");
        break;
      case 7:
        Scope(c, g.cls, ls),
        ck(tn::launch_root_grouped(reinterpret_cast<tn::RootDesc*>(d), g.count, int(g.p0), guard_mode,
                                   ls),
           "grouped root");
        break;
      case 8: {
        const Bucket& bk = bks[size_t(g.p0)];
        const tn::Step& st = bk.P->steps[size_t(g.p1)];
        int maxD = 1;
        for (int k = 0; k < st.n; ++k) maxD = std::max(maxD, st.D[k]);
        Scope(c, TN_KC_CLOSE, ls),
        ck(tn::launch_close_f32(ws[size_t(g.p0)].Y, ws[size_t(g.p0)].sY,
                                bk.tabs[size_t(g.p1)].y_off, bk.tabs[size_t(g.p1)].D, st.n, maxD,
                                res_logscale + bk.res_off, res_logz + bk.res_off,
                                res_status + bk.res_off, int(bk.idx.size()), ls),
           "close");
        break;
      }
      default:
        fail(TN_ERR_INVALID, "grouped launch kind");
    }
    if (guard_mode) {
      const std::string at = "guard: launch " + std::to_string(li) + " of " +
                             std::to_string(gb.launches.size()) + " kind " +
                             std::to_string(g.kind) + " count " + std::to_string(g.count) +
                             " extents " + std::to_string(g.p0) + "," + std::to_string(g.p1) +
                             "," + std::to_string(g.p2);
      const cudaError_t e = cudaStreamSynchronize(strm);
      if (e != cudaSuccess) fail(TN_ERR_CUDA, at + ": " + cudaGetErrorString(e));
      unsigned long long rec[4] = {0, 0, 0, 0};
      ck(cudaMemcpy(rec, grec, sizeof(rec), cudaMemcpyDeviceToHost), "guard: read record");
      if (rec[0]) {
        char tag[32];
        std::snprintf(tag, sizeof(tag), "0x%llx", rec[0] - 1);
        std::string m = at + ": access tag " + tag + " block " + std::to_string(rec[1]) +
                        " value/address " + std::to_string(rec[2]) + " bytes/limit " +
                        std::to_string(rec[3]) + " at " + where(rec[2]);
        if (g.kind == 2 || g.kind == 3) {
          const long long gx = (g.p1 + 63) / 64, gy = (g.p0 + 63) / 64;
          const long long q = (long long)(rec[1] / (unsigned long long)(gx * gy));
          if (q < g.count) {
            const tn::GemmDesc x = reinterpret_cast<const tn::GemmDesc*>(gb.bytes.data() + g.off)[q];
            auto ad = [](const void* v) { return (unsigned long long)reinterpret_cast<uintptr_t>(v); };
            m += "; problem " + std::to_string(q) + " M " + std::to_string(x.M) + " N " +
                 std::to_string(x.N) + " K " + std::to_string(x.K) + " lda " +
                 std::to_string(x.lda) + " ldb " + std::to_string(x.ldb) + " ldc " +
                 std::to_string(x.ldc) + " ldct " + std::to_string(x.ldct) + " ct_cols " +
                 std::to_string(x.ct_cols) + " A at " + where(ad(x.A)) + " B at " +
                 where(ad(x.B)) + " C at " + where(ad(x.C)) +
                 (x.Ct ? " Ct at " + where(ad(x.Ct)) : std::string());
          }
        }
        fail(TN_ERR_INVALID, m);
      }
    }
  }
}

constexpr size_t kPoolStreams = 8;  // concurrent buckets of one batch

// Restores the ctx's result pointers after a bucketed batch (also on error).
struct ResultView {
  tn_ctx* c;
  double *logz, *logscale;
  int* status;
  explicit ResultView(tn_ctx* c_) : c(c_), logz(c_->logz), logscale(c_->logscale), status(c_->status) {}
  void at(size_t off) {
    c->logz = logz + off;
    c->logscale = logscale + off;
    c->status = status + off;
  }
  ~ResultView() {
    c->logz = logz;
    c->logscale = logscale;
    c->status = status;
  }
};

// Algorithm partitioned_contract for a batch whose instances may have
// different plans (sizes, chi): instances with structurally equal plans form
// a bucket; all buckets' tables go to the device in one copy, the workspace
// is sized for the largest bucket and reused by the next (stream order), and
// each bucket writes its slice of the results.  upload = false leaves the
// tables as a previous identical call placed them (graph capture).
void run_batch(tn_ctx* c, const tn_plan_t* const* plans, int n, const double* const* sites,
               int precision, bool learned, cudaStream_t strm, bool upload) {
  const bool tc = precision != TN_PREC_FP64;
  const int sub_split = (precision == TN_PREC_TF32_FAST) ? 0 : 1;
  const bool factored = precision == TN_PREC_TF32;
  std::vector<Bucket> bks;
  for (int i = 0; i < n; ++i) {
    size_t b = bks.size();
    for (size_t j = 0; j < bks.size(); ++j)
      if (tn::plans_equivalent(bks[j].P, plans[i])) {
        b = j;
        break;
      }
    if (b == bks.size()) {
      bks.emplace_back();
      bks.back().P = plans[i];
    }
    bks[b].idx.push_back(i);
    bks[b].sites.push_back(sites[i]);
  }
  if (learned && bks.size() > 1)
    fail(TN_ERR_UNSUPPORTED, "learned ranks need one plan structure per batch");
  size_t ws_max = 0, ws_sum = 0, tab_tot = 0, res = 0;
  std::vector<int> slot(n, 0);
  for (Bucket& bk : bks) {
    const int B = int(bk.idx.size());
    for (const tn::Step& st : bk.P->steps) bk.lay.push_back(tc ? lay_f32(st) : lay_fp64(st));
    if (tc)
      carve_f32(c, bk.P, bk.lay, B, true, &bk.ws_bytes);
    else
      carve(c, plan_dims(bk.P), B, bk.P->n_vertices, true, &bk.ws_bytes);
    ws_max = std::max(ws_max, bk.ws_bytes);
    bk.ws_off = ws_sum;
    ws_sum += align256(bk.ws_bytes);
    bk.tab_off = tab_tot;
    tab_tot += align256(tables_bytes(bk.P, B));
    bk.res_off = res;
    for (int k = 0; k < B; ++k) slot[bk.idx[k]] = int(res) + k;
    res += B;
  }
  ensure_results(c, n);
  // several buckets run concurrently on a pool of streams, each in a
  // workspace slice of its own (the learned ranks keep one bucket)
  const int nstreams = bks.size() > 1 ? int(std::min<size_t>(bks.size(), kPoolStreams)) : 0;
  if (nstreams) {
    char* wbase = static_cast<char*>(c->arena.get(ws_sum));
    for (Bucket& bk : bks) bk.ws_at = wbase + bk.ws_off;
    while (int(c->pool.size()) < nstreams) {
      cudaStream_t ps = nullptr;
      ck(cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking), "cudaStreamCreate");
      c->pool.push_back(ps);
      cudaEvent_t ev = nullptr;
      ck(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "cudaEventCreate");
      c->joins.push_back(ev);
    }
    if (!c->fork) ck(cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming), "cudaEventCreate");
  } else {
    c->arena.get(ws_max);
  }
  char* dbase = static_cast<char*>(c->tables.get(tab_tot));
  char* h = upload ? static_cast<char*>(pinned_get(c, tab_tot)) : nullptr;
  for (Bucket& bk : bks)
    bk.tabs = fill_tables(bk.P, bk.lay, bk.sites.data(), int(bk.idx.size()),
                          h ? h + bk.tab_off : nullptr, dbase + bk.tab_off, &bk.tens_table,
                          &bk.off_dev, &bk.len_dev);
  if (upload) {
    ck(cudaMemcpyAsync(dbase, h, tab_tot, cudaMemcpyHostToDevice, strm), "upload tables");
    ck(cudaEventRecord(c->pinned_free, strm), "cudaEventRecord");
  }
  ck(cudaMemsetAsync(c->err_flag, 0, 2 * sizeof(int), strm), "memset err");
  {
    ResultView view(c);
    if (nstreams) {
      ck(cudaEventRecord(c->fork, strm), "cudaEventRecord");
      for (int q = 0; q < nstreams; ++q)
        ck(cudaStreamWaitEvent(c->pool[q], c->fork, 0), "cudaStreamWaitEvent");
    }
    // largest buckets first, dealt round-robin over the streams
    std::vector<size_t> order(bks.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](size_t a, size_t b) { return bks[a].ws_bytes > bks[b].ws_bytes; });
    const bool grouped = tc && c->grouped && !learned && bks.size() > kPoolStreams &&
                         grouped_eligible(bks);
    if (grouped) {
      run_grouped_tc(c, bks, factored, upload, view.logz, view.logscale, view.status, strm);
    } else {
      for (size_t j = 0; j < order.size(); ++j) {
        const Bucket& bk = bks[order[j]];
        cudaStream_t bs = nstreams ? c->pool[j % nstreams] : strm;
        view.at(bk.res_off);
        if (tc)
          run_plan_tc(c, bk, sub_split, factored, learned, bs);
        else
          run_plan(c, bk, precision, learned, bs);
      }
    }
    if (nstreams)
      for (int q = 0; q < nstreams; ++q) {
        ck(cudaEventRecord(c->joins[q], c->pool[q]), "cudaEventRecord");
        ck(cudaStreamWaitEvent(strm, c->joins[q], 0), "cudaStreamWaitEvent");
      }
  }
  c->slot = std::move(slot);
  c->slot_identity = bks.size() == 1;
  c->stream = strm;
  c->last_batch = n;
  c->pending = true;
  c->wait_probe = false;
}

template <class F>
tn_status guarded(tn_ctx* c, const char* fn, F&& f) {
  try {
    f();
  } catch (const Fail& e) {
    const std::string m = std::string(fn) + ": " + e.msg;
    if (c) c->err = m;
    tn::set_error(m);
    return e.st;
  } catch (const std::bad_alloc&) {
    const std::string m = std::string(fn) + ": host allocation failed";
    if (c) c->err = m;
    tn::set_error(m);
    return TN_ERR_OOM;
  } catch (...) {
    const std::string m = std::string(fn) + ": unexpected error";
    if (c) c->err = m;
    tn::set_error(m);
    return TN_ERR_INVALID;
  }
  return TN_OK;
}

}  // namespace

extern "C" tn_status tn_ctx_create(int32_t device, tn_ctx_t** out) {
  if (!out) {
    tn::set_error("tn_ctx_create: out is NULL");
    return TN_ERR_INVALID;
  }
  *out = nullptr;
  tn_ctx* c = new (std::nothrow) tn_ctx();
  if (!c) {
    tn::set_error("tn_ctx_create: host allocation failed");
    return TN_ERR_OOM;
  }
  tn_status s = guarded(nullptr, "tn_ctx_create", [&] {
    int n = 0;
    ck(cudaGetDeviceCount(&n), "cudaGetDeviceCount");
    if (device < 0 || device >= n) fail(TN_ERR_INVALID, "device ordinal out of range");
    ck(cudaSetDevice(device), "cudaSetDevice");
    c->device = device;
    ck(cudaEventCreateWithFlags(&c->pinned_free, cudaEventDisableTiming), "cudaEventCreate");
    ck(tn::eigh_configure(), "eigh configure");
    int major = 0, minor = 0;
    ck(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device), "attribute");
    ck(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device), "attribute");
    c->tc_ready = (major == 10 && minor == 3) && tn::tc_gemm_configure() == cudaSuccess &&
                  tn::svd_configure() == cudaSuccess;
    cudaGetLastError();
  });
  if (s != TN_OK) {
    delete c;
    return s;
  }
  *out = c;
  return TN_OK;
}

extern "C" tn_status tn_ctx_destroy(tn_ctx_t* c) {
  if (!c) return TN_OK;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  c->arena.release();
  c->stage.release();
  c->tables.release();
  c->results.release();
  c->model_buf.release();
  c->learn_buf.release();
  c->train_buf.release();
  c->aux_buf.release();
  c->judge_buf.release();
  if (c->pinned) cudaFreeHost(c->pinned);
  if (c->pinned_free) cudaEventDestroy(c->pinned_free);
  for (cudaStream_t ps : c->pool) cudaStreamDestroy(ps);
  for (cudaEvent_t ev : c->joins) cudaEventDestroy(ev);
  if (c->fork) cudaEventDestroy(c->fork);
  if (c->gready) cudaEventDestroy(c->gready);
  delete c;
  return TN_OK;
}

extern "C" tn_status tn_contract_approx(tn_ctx_t* c, const tn_plan_t* const* plans, int32_t n_inst,
                                        const double* const* sites_dev, int32_t precision,
                                        int32_t learned_chi, void* stream) {
  if (!c) {
    tn::set_error("tn_contract_approx: ctx is NULL");
    return TN_ERR_INVALID;
  }
  return guarded(c, "tn_contract_approx", [&] {
    if (!plans || !sites_dev || n_inst < 1) fail(TN_ERR_INVALID, "plans/sites NULL or n_inst < 1");
    if (learned_chi && !c->have_model)
      fail(TN_ERR_INVALID, "learned_chi = 1 or 2 needs a rank model (tn_rank_model_load)");
    if (learned_chi < 0 || learned_chi > 2) fail(TN_ERR_INVALID, "learned_chi must be 0, 1 or 2");
    if (learned_chi)
      for (int i = 1; i < n_inst; ++i)
        if (plans[i] && !tn::plans_equivalent(plans[0], plans[i]))
          fail(TN_ERR_UNSUPPORTED, "learned ranks need one plan structure per batch");
    for (int i = 0; i < n_inst; ++i)
      if (!plans[i] || !sites_dev[i]) fail(TN_ERR_INVALID, "NULL plan or site buffer");
    ck(cudaSetDevice(c->device), "cudaSetDevice");
    cudaStream_t strm = static_cast<cudaStream_t>(stream);
    if (precision == TN_PREC_TF32 || precision == TN_PREC_TF32_FAST ||
        precision == TN_PREC_TF32_GRAM) {
      if (!c->tc_ready) fail(TN_ERR_UNSUPPORTED, "tcgen05 path unavailable on this device");
    } else if (precision != TN_PREC_FP64) {
      fail(TN_ERR_UNSUPPORTED, "precision mode not implemented in this build");
    }
    if (learned_chi == 2) {
      // the uniform-chi judge: a run at min(chi_uniform, r_v), then the
      // learned run; per instance the smaller summed discarded share wins
      const size_t nb = size_t(n_inst);
      char* jb = static_cast<char*>(c->judge_buf.get(4 * align256(sizeof(double) * nb) +
                                                      2 * align256(sizeof(int) * nb)));
      double* acc_l = reinterpret_cast<double*>(jb);
      double* acc_u = reinterpret_cast<double*>(jb + align256(sizeof(double) * nb));
      double* logz_u = reinterpret_cast<double*>(jb + 2 * align256(sizeof(double) * nb));
      int* status_u = reinterpret_cast<int*>(jb + 3 * align256(sizeof(double) * nb));
      int* used = status_u + align256(sizeof(int) * nb) / sizeof(int);
      struct Reset {
        tn_ctx* c;
        ~Reset() {
          c->hook_fixed_chi = 0;
          c->hook_acc = nullptr;
        }
      } reset{c};
      c->hook_fixed_chi = c->chi_uniform;
      c->hook_acc = acc_u;
      run_batch(c, plans, n_inst, sites_dev, precision, false, strm, true);
      ck(cudaMemcpyAsync(logz_u, c->logz, sizeof(double) * nb, cudaMemcpyDeviceToDevice, strm),
         "copy logz");
      ck(cudaMemcpyAsync(status_u, c->status, sizeof(int) * nb, cudaMemcpyDeviceToDevice, strm),
         "copy status");
      c->hook_fixed_chi = 0;
      c->hook_acc = c->rec_acc ? nullptr : acc_l;
      run_batch(c, plans, n_inst, sites_dev, precision, true, strm, true);
      ck(tn::launch_judge_select(c->rec_acc ? c->rec_acc : acc_l, acc_u, logz_u, status_u,
                                 c->logz, c->status, used, n_inst, strm),
         "judge");
      c->judged = used;
      c->judged_n = n_inst;
    } else {
      run_batch(c, plans, n_inst, sites_dev, precision, learned_chi != 0, strm, true);
      c->judged = nullptr;
    }
  });
}

extern "C" tn_status tn_rank_judged(tn_ctx_t* c, int32_t* used_learned_host, int32_t n_inst) {
  if (!c) {
    tn::set_error("tn_rank_judged: ctx is NULL");
    return TN_ERR_INVALID;
  }
  return guarded(c, "tn_rank_judged", [&] {
    if (!used_learned_host || !c->judged || n_inst != c->judged_n)
      fail(TN_ERR_INVALID, "no judged batch of this size (learned_chi = 2) has run");
    ck(cudaSetDevice(c->device), "cudaSetDevice");
    ck(cudaMemcpyAsync(used_learned_host, c->judged, sizeof(int) * n_inst,
                       cudaMemcpyDeviceToHost, c->stream),
       "copy judged");
    ck(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  });
}

extern "C" int32_t tn_rank_model_params(void) { return tn::rank_model_params(); }

extern "C" tn_status tn_rank_model_load(tn_ctx_t* c, const float* weights_host, int32_t n_params,
                                        int32_t chi_uniform) {
  if (!c) {
    tn::set_error("tn_rank_model_load: ctx is NULL");
    return TN_ERR_INVALID;
  }
  return guarded(c, "tn_rank_model_load", [&] {
    if (!weights_host) {
      c->have_model = false;
      return;
    }
    const int np = tn::rank_model_params();
    if (n_params != np) fail(TN_ERR_INVALID, "n_params differs from tn_rank_model_params()");
    if (chi_uniform < 1) fail(TN_ERR_INVALID, "chi_uniform must be >= 1");
    ck(cudaSetDevice(c->device), "cudaSetDevice");
    float* tmp = static_cast<float*>(c->train_buf.get(sizeof(float) * size_t(np)));
    void* bf = c->model_buf.get(2 * size_t(np));
    ck(cudaMemcpy(tmp, weights_host, sizeof(float) * size_t(np), cudaMemcpyHostToDevice),
       "copy weights");
    ck(tn::launch_to_bf16(tmp, bf, np, nullptr), "to bf16");
    ck(cudaDeviceSynchronize(), "synchronize");
    c->chi_uniform = chi_uniform;
    c->have_model = true;
  });
}

extern "C" tn_status tn_rank_record(tn_ctx_t* c, float* feat_dev, double* spec_dev,
                                    int32_t* chi_dev, double* acc_dev, int64_t cap_edges) {
  if (!c) {
    tn::set_error("tn_rank_record: ctx is NULL");
    return TN_ERR_INVALID;
  }
  return guarded(c, "tn_rank_record", [&] {
    if (cap_edges < 0) fail(TN_ERR_INVALID, "cap_edges < 0");
    c->rec_feat = feat_dev;
    c->rec_spec = spec_dev;
    c->rec_chi = chi_dev;
    c->rec_acc = acc_dev;
    c->rec_cap = cap_edges;
  });
}

extern "C" tn_status tn_rank_labels(tn_ctx_t* c, const double* spec_dev, int32_t n_inst,
                                    const int32_t* cap, const int32_t* pass_start,
                                    int32_t n_pass, int32_t chi_uniform, int32_t* chi_dev,
                                    float* feat_dev, void* stream) {
  if (!c) {
    tn::set_error("tn_rank_labels: ctx is NULL");
    return TN_ERR_INVALID;
  }
  return guarded(c, "tn_rank_labels", [&] {
    if (!spec_dev || !cap || !pass_start || !chi_dev || n_inst < 1 || n_pass < 1 ||
        n_pass > 65535 || chi_uniform < 1)
      fail(TN_ERR_INVALID, "invalid argument");
    if (pass_start[0] != 0) fail(TN_ERR_INVALID, "pass_start[0] must be 0");
    for (int p = 0; p < n_pass; ++p) {
      const int ne = pass_start[p + 1] - pass_start[p];
      if (ne < 1 || ne > tn::water_fill_max_edges())
        fail(TN_ERR_INVALID, "a pass needs 1 .. 256 edges");
    }
    const int n_edges = pass_start[n_pass];
    for (int e = 0; e < n_edges; ++e)
      if (cap[e] < 1) fail(TN_ERR_INVALID, "cap entries must be >= 1");
    ck(cudaSetDevice(c->device), "cudaSetDevice");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // [cap (n_edges) | pass_start (n_pass + 1)]
    std::vector<int32_t> h;
    h.insert(h.end(), cap, cap + n_edges);
    h.insert(h.end(), pass_start, pass_start + n_pass + 1);
    int32_t* d = static_cast<int32_t*>(c->aux_buf.get(sizeof(int32_t) * h.size()));
    ck(cudaMemcpyAsync(d, h.data(), sizeof(int32_t) * h.size(), cudaMemcpyHostToDevice, st),
       "copy label tables");
    ck(tn::launch_water_fill(spec_dev, d, d + n_edges, chi_uniform, n_pass, n_inst, chi_dev,
                             feat_dev, st),
       "water fill");
    ck(cudaStreamSynchronize(st), "cudaStreamSynchronize");
  });
}

extern "C" tn_status tn_rank_model_grad(tn_ctx_t* c, const float* X_dev, const float* y_dev,
                                        const int32_t* idx_dev, int32_t n, const float* w_dev,
                                        float* grad_dev, float* loss_dev, void* stream) {
  if (!c) {
    tn::set_error("tn_rank_model_grad: ctx is NULL");
    return TN_ERR_INVALID;
  }
  return guarded(c, "tn_rank_model_grad", [&] {
    if (!X_dev || !y_dev || !w_dev || !grad_dev || !loss_dev || n < 1)
      fail(TN_ERR_INVALID, "invalid argument");
    ck(cudaSetDevice(c->device), "cudaSetDevice");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int np = tn::rank_model_params();
    if (!idx_dev) {
      int* iota = static_cast<int*>(c->aux_buf.get(sizeof(int) * size_t(n)));
      ck(tn::launch_iota(iota, n, st), "iota");
      idx_dev = iota;
    }
    ck(cudaMemsetAsync(grad_dev, 0, sizeof(float) * size_t(np), st), "memset grad");
    ck(cudaMemsetAsync(loss_dev, 0, sizeof(float), st), "memset loss");
    ck(tn::launch_mlp_grad(X_dev, y_dev, idx_dev, n, 1.f / float(n), w_dev, grad_dev, loss_dev,
                           st),
       "mlp grad");
  });
}

extern "C" tn_status tn_rank_model_train(tn_ctx_t* c, const float* X_dev, const float* y_dev,
                                         const int32_t* idx_dev, int32_t steps, int32_t batch,
                                         float lr, float* w_dev, float* loss_dev, void* stream) {
  if (!c) {
    tn::set_error("tn_rank_model_train: ctx is NULL");
    return TN_ERR_INVALID;
  }
  return guarded(c, "tn_rank_model_train", [&] {
    if (!X_dev || !y_dev || !idx_dev || !w_dev || !loss_dev || steps < 1 || batch < 1 ||
        !(lr > 0.f))
      fail(TN_ERR_INVALID, "invalid argument");
    ck(cudaSetDevice(c->device), "cudaSetDevice");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int np = tn::rank_model_params();
    float* g = static_cast<float*>(c->train_buf.get(3 * sizeof(float) * size_t(np)));
    float* m = g + np;
    float* v = m + np;
    ck(cudaMemsetAsync(g, 0, 3 * sizeof(float) * size_t(np), st), "memset adam");
    ck(cudaMemsetAsync(loss_dev, 0, sizeof(float) * size_t(steps), st), "memset loss");
    for (int t = 0; t < steps; ++t) {
      ck(tn::launch_mlp_grad(X_dev, y_dev, idx_dev + (long long)t * batch, batch,
                             1.f / float(batch), w_dev, g, loss_dev + t, st),
         "mlp grad");
      ck(tn::launch_adam(w_dev, g, m, v, np, lr, 0.9f, 0.999f, 1e-8f, t + 1, st), "adam");
    }
  });
}

extern "C" tn_status tn_logz(tn_ctx_t* c, double* logz_host, int32_t* status_host, int32_t n_inst) {
  if (!c) {
    tn::set_error("tn_logz: ctx is NULL");
    return TN_ERR_INVALID;
  }
  tn_status first = TN_OK;
  tn_status s = guarded(c, "tn_logz", [&] {
    if (!c->pending) fail(TN_ERR_INVALID, "no batch has been launched");
    if (n_inst != c->last_batch) fail(TN_ERR_INVALID, "n_inst differs from the launched batch");
    if (!logz_host || !status_host) fail(TN_ERR_INVALID, "NULL output");
    ck(cudaSetDevice(c->device), "cudaSetDevice");
    // bucketed batches keep results in slot order: copy, then put back in
    // instance order
    const bool ident = c->slot_identity || int(c->slot.size()) != n_inst;
    std::vector<double> lz(ident ? 0 : n_inst);
    std::vector<int> stt(ident ? 0 : n_inst);
    double* lz_dst = ident ? logz_host : lz.data();
    int* st_dst = ident ? status_host : stt.data();
    ck(cudaMemcpyAsync(lz_dst, c->logz, sizeof(double) * n_inst, cudaMemcpyDeviceToHost,
                       c->stream),
       "copy logz");
    ck(cudaMemcpyAsync(st_dst, c->status, sizeof(int) * n_inst, cudaMemcpyDeviceToHost,
                       c->stream),
       "copy status");
    int err = 0;
    ck(cudaMemcpyAsync(&err, c->err_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream),
       "copy err");
    ck(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    if (!ident)
      for (int i = 0; i < n_inst; ++i) {
        logz_host[i] = lz[c->slot[i]];
        status_host[i] = stt[c->slot[i]];
      }
    if (err) {
      for (int i = 0; i < n_inst; ++i) {
        status_host[i] = TN_ERR_TIMEOUT;
        logz_host[i] = NAN;
      }
    }
    for (int i = 0; i < n_inst; ++i)
      if (status_host[i] != TN_OK && first == TN_OK) first = tn_status(status_host[i]);
    if (first != TN_OK) {
      c->err = "tn_logz: instance failed with status " + std::to_string(int(first));
      tn::set_error(c->err);
    }
  });
  return s != TN_OK ? s : first;
}

extern "C" tn_status tn_contract_approx_host(tn_ctx_t* c, const tn_plan_t* const* plans,
                                             int32_t n_inst, const double* const* sites_host,
                                             int32_t precision, int32_t learned_chi,
                                             double* logz_host, int32_t* status_host,
                                             void* stream) {
  if (!c) {
    tn::set_error("tn_contract_approx_host: ctx is NULL");
    return TN_ERR_INVALID;
  }
  tn_status s = guarded(c, "tn_contract_approx_host", [&] {
    if (!plans || !sites_host || n_inst < 1 || !plans[0])
      fail(TN_ERR_INVALID, "plans/sites NULL or n_inst < 1");
    ck(cudaSetDevice(c->device), "cudaSetDevice");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // each instance's site buffer at its own offset (plans may differ)
    std::vector<int64_t> off(n_inst + 1, 0);
    for (int i = 0; i < n_inst; ++i) {
      if (!plans[i] || !sites_host[i]) fail(TN_ERR_INVALID, "NULL plan or site buffer");
      off[i + 1] = off[i] + ((plans[i]->site_elems + 31) & ~int64_t(31));
    }
    double* dev = static_cast<double*>(c->stage.get(sizeof(double) * size_t(off[n_inst])));
    std::vector<const double*> ptrs(n_inst);
    for (int i = 0; i < n_inst; ++i) {
      ck(cudaMemcpyAsync(dev + off[i], sites_host[i], sizeof(double) * plans[i]->site_elems,
                         cudaMemcpyHostToDevice, st),
         "copy sites");
      ptrs[i] = dev + off[i];
    }
    tn_status r = tn_contract_approx(c, plans, n_inst, ptrs.data(), precision, learned_chi, stream);
    if (r != TN_OK) fail(r, c->err);
  });
  if (s != TN_OK) return s;
  return tn_logz(c, logz_host, status_host, n_inst);
}

namespace {
// One factored mixed-precision pass on explicit FP64 blocks (tn_embed_tree
// with TN_PREC_TF32): blocks converted to the FP32 layout (with the
// transposed copies the tensor-core contractions read), dm_pass_tc, and the
// tree tensors converted back to the caller's packed FP64 layout.
void embed_tree_tc(tn_ctx* c, const tn::Step& st, const tn_plan_t* tmp, int B,
                   const double* const* blocks_dev, double* const* tree_dev, double* lognorm_dev,
                   int32_t* status_dev, cudaStream_t strm) {
  const int n = st.n;
  const std::vector<Lay> lay{lay_f32(st)};
  const Lay& l = lay[0];
  ensure_results(c, B);
  const WsF w = carve_f32(c, tmp, lay, B);
  // tables: block pointers, tree pointers, conversion segments, R_k offsets and D
  const size_t o_in = 0, o_out = align256(sizeof(void*) * B);
  const size_t o_seg_in = o_out + align256(sizeof(void*) * B);
  const size_t o_seg_out = o_seg_in + align256(sizeof(tn::CvtSeg) * n);
  const size_t o_roff = o_seg_out + align256(sizeof(tn::CvtSeg) * n);
  const size_t o_D = o_roff + align256(sizeof(int64_t) * n);
  const size_t tot = o_D + align256(sizeof(int32_t) * (n + 1));
  char* h = static_cast<char*>(pinned_get(c, tot));
  char* d = static_cast<char*>(c->tables.get(tot));
  std::memcpy(h + o_in, blocks_dev, sizeof(void*) * B);
  std::memcpy(h + o_out, tree_dev, sizeof(void*) * B);
  tn::CvtSeg* si = reinterpret_cast<tn::CvtSeg*>(h + o_seg_in);
  tn::CvtSeg* so = reinterpret_cast<tn::CvtSeg*>(h + o_seg_out);
  int max_in = 1, max_out = 1;
  int64_t out_pos = 0;
  for (int k = 0; k < n; ++k) {
    const int rows = st.site[k].a, cols = st.d[k] * st.D[k];
    si[k] = tn::CvtSeg{st.y_off[k], l.y_off[k], rows, cols};
    max_in = std::max(max_in, rows * cols);
  }
  for (int k = 1; k < n; ++k) {  // tree tensors U_1 .. U_{n-2}, then the root
    const int64_t sz = st.s_size[k];
    so[k - 1] = tn::CvtSeg{l.s_off[k], out_pos, 1, int32_t(sz)};
    out_pos += sz;
    max_out = std::max<int>(max_out, int(sz));
  }
  std::vector<int64_t> ro(l.r_off);
  ro.resize(n, 0);
  std::memcpy(h + o_roff, ro.data(), sizeof(int64_t) * n);
  std::vector<int32_t> Dv(st.D);
  int mx = 1;
  for (int x : Dv) mx = std::max(mx, x);
  Dv.push_back(mx);
  std::memcpy(h + o_D, Dv.data(), sizeof(int32_t) * (n + 1));
  ck(cudaMemcpyAsync(d, h, tot, cudaMemcpyHostToDevice, strm), "upload tables");
  ck(cudaEventRecord(c->pinned_free, strm), "cudaEventRecord");
  ck(cudaMemsetAsync(c->logscale, 0, sizeof(double) * B, strm), "memset");
  ck(cudaMemsetAsync(c->status, 0, sizeof(int) * B, strm), "memset");
  ck(cudaMemsetAsync(c->err_flag, 0, 2 * sizeof(int), strm), "memset err");
  ck(tn::launch_convert_segments_d2f(reinterpret_cast<const double* const*>(d + o_in), w.Y, w.sY,
                                     w.Yt, reinterpret_cast<const tn::CvtSeg*>(d + o_seg_in), n,
                                     max_in, B, strm),
     "convert blocks");
  StepTables tab{};
  tab.r_off = reinterpret_cast<int64_t*>(d + o_roff);
  tab.D = reinterpret_cast<int32_t*>(d + o_D);
  dm_pass_tc(c, st, l, w, w.S1, B, 1, true, &tab, strm);
  ck(tn::launch_convert_segments_f2d(w.S1, w.sS, reinterpret_cast<double* const*>(d + o_out),
                                     reinterpret_cast<const tn::CvtSeg*>(d + o_seg_out), n - 1,
                                     max_out, B, strm),
     "convert tree");
  ck(cudaMemcpyAsync(lognorm_dev, c->logscale, sizeof(double) * B, cudaMemcpyDeviceToDevice,
                     strm),
     "copy lognorm");
  ck(cudaMemcpyAsync(status_dev, c->status, sizeof(int) * B, cudaMemcpyDeviceToDevice, strm),
     "copy status");
}
}  // namespace

extern "C" tn_status tn_embed_tree(tn_ctx_t* c, int32_t n_inst, int32_t n_legs,
                                   const int32_t* leg_dim, const int32_t* bond_dim,
                                   const double* const* blocks_dev, int32_t chi,
                                   const int32_t* chi_per_edge, int32_t precision,
                                   double* const* tree_dev, double* lognorm_dev,
                                   int32_t* status_dev, int32_t* ranks_host, void* stream) {
  if (!c) {
    tn::set_error("tn_embed_tree: ctx is NULL");
    return TN_ERR_INVALID;
  }
  return guarded(c, "tn_embed_tree", [&] {
    if (n_inst < 1 || n_legs < 3 || !leg_dim || !bond_dim || !blocks_dev || !tree_dev ||
        !lognorm_dev || !status_dev || !ranks_host)
      fail(TN_ERR_INVALID, "invalid argument");
    if (chi < 1 && !chi_per_edge) fail(TN_ERR_INVALID, "chi must be >= 1");
    if (precision != TN_PREC_FP64 && precision != TN_PREC_TF32)
      fail(TN_ERR_UNSUPPORTED, "tn_embed_tree runs TN_PREC_FP64 or TN_PREC_TF32");
    if (precision == TN_PREC_TF32 && !c->tc_ready)
      fail(TN_ERR_UNSUPPORTED, "tcgen05 path unavailable on this device");
    const int n = n_legs;
    tn::Step st;
    st.kind = 1;
    st.n = n;
    st.d.assign(leg_dim, leg_dim + n);
    st.D.assign(n, 1);
    for (int k = 0; k < n; ++k) {
      if (st.d[k] < 1) fail(TN_ERR_INVALID, "leg dim < 1");
      if (k < n - 1) {
        st.D[k] = bond_dim[k];
        if (st.D[k] < 1 || st.D[k] > (1 << 16)) fail(TN_ERR_INVALID, "bond dim out of range");
      }
    }
    st.site.resize(n);
    for (int k = 0; k < n; ++k) {
      tn::SiteOp o{};
      o.a = (k == 0) ? 1 : st.D[k - 1];
      o.b = st.D[k];
      o.dp = o.dhl = o.dhr = 1;
      o.de = st.d[k];
      st.site[k] = o;
    }
    st.r.assign(n - 1, 0);
    st.r[0] = st.d[0];
    for (int k = 1; k <= n - 2; ++k) {
      double beyond = 1;
      for (int j = k + 1; j < n; ++j) beyond *= st.d[j];
      const int ck_ = chi_per_edge ? chi_per_edge[k] : chi;
      if (ck_ < 1) fail(TN_ERR_INVALID, "chi_per_edge entries must be >= 1");
      double r = std::min<double>(ck_, double(st.r[k - 1]) * st.d[k]);
      r = std::min<double>(r, st.D[k]);
      r = std::min<double>(r, beyond);
      st.r[k] = int(r);
    }
    // layouts identical to the planner's
    st.y_off.assign(n, 0);
    long long off = 0;
    for (int k = 0; k < n; ++k) {
      st.y_off[k] = off;
      off += (long long)st.site[k].a * st.d[k] * st.D[k];
    }
    st.y_total = off;
    st.s_off.assign(n, 0);
    st.s_size.assign(n, 0);
    off = 0;
    for (int k = 0; k < n; ++k) {
      const long long left = (k == 0) ? 1 : st.r[k - 1];
      const long long right = (k == n - 1) ? 1 : st.r[k];
      st.s_off[k] = off;
      st.s_size[k] = left * st.d[k] * right;
      off += st.s_size[k];
    }
    st.s_total = off;
    st.r_off.assign(n, 0);
    off = 0;
    for (int k = 1; k <= n - 1; ++k) {
      st.r_off[k] = off;
      off += (long long)st.D[k] * st.D[k];
    }
    st.r_total = off;
    tn_plan_t tmp;
    tmp.steps.push_back(st);
    ck(cudaSetDevice(c->device), "cudaSetDevice");
    cudaStream_t strm = static_cast<cudaStream_t>(stream);
    if (precision == TN_PREC_TF32) {
      for (int k = 1; k <= n - 2; ++k)
        if (!tn::svd_left_supported(st.r[k - 1] * st.d[k], st.D[k], st.r[k]))
          fail(TN_ERR_UNSUPPORTED,
               "TN_PREC_TF32 needs dim A_v <= 128, tree-edge dims <= 128 and ranks <= 64");
      embed_tree_tc(c, st, &tmp, n_inst, blocks_dev, tree_dev, lognorm_dev, status_dev, strm);
      for (int k = 0; k < n - 1; ++k) ranks_host[k] = st.r[k];
      return;
    }
    const Dims dm = plan_dims(&tmp);
    ensure_results(c, n_inst);
    const Ws w = carve(c, dm, n_inst, 1);
    ck(cudaMemsetAsync(c->logscale, 0, sizeof(double) * n_inst, strm), "memset");
    ck(cudaMemsetAsync(c->status, 0, sizeof(int) * n_inst, strm), "memset");
    for (int i = 0; i < n_inst; ++i)
      ck(cudaMemcpyAsync(w.Y + w.sY * i, blocks_dev[i], sizeof(double) * st.y_total,
                         cudaMemcpyDeviceToDevice, strm),
         "copy blocks");
    dm_pass(c, st, w, w.S1, n_inst, precision, strm);
    for (int i = 0; i < n_inst; ++i)
      ck(cudaMemcpyAsync(tree_dev[i], w.S1 + w.sS * i + st.s_off[1],
                         sizeof(double) * (st.s_total - st.s_size[0]), cudaMemcpyDeviceToDevice,
                         strm),
         "copy tree");
    ck(cudaMemcpyAsync(lognorm_dev, c->logscale, sizeof(double) * n_inst,
                       cudaMemcpyDeviceToDevice, strm),
       "copy lognorm");
    ck(cudaMemcpyAsync(status_dev, c->status, sizeof(int) * n_inst, cudaMemcpyDeviceToDevice,
                       strm),
       "copy status");
    for (int k = 0; k < n - 1; ++k) ranks_host[k] = st.r[k];
  });
}

// ------------------------------------------------ allocation-free variant
// Workspace of tn_embed_tree_noalloc: a fixed device array compiled into the
// library (every device that loads the library holds it until exit).  Host
// code must not pass the symbol itself to a kernel; its device address is
// looked up once per device with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[TN_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices] = {};
}  // namespace

extern "C" tn_status tn_embed_tree_noalloc(int32_t n_inst, int32_t n_legs, const int32_t* leg_dim,
                                           const int32_t* bond_dim,
                                           const double* const* blocks_dev, int32_t chi,
                                           const int32_t* chi_per_edge, double* const* tree_dev,
                                           double* lognorm_dev, int32_t* status_dev,
                                           int32_t* ranks_host, void* stream) {
  return guarded(nullptr, "tn_embed_tree_noalloc", [&] {
    if (n_inst < 1 || n_legs < 3 || !leg_dim || !bond_dim || !blocks_dev || !tree_dev ||
        !lognorm_dev || !status_dev || !ranks_host)
      fail(TN_ERR_INVALID, "invalid argument");
    if (chi < 1 && !chi_per_edge) fail(TN_ERR_INVALID, "chi must be >= 1");
    const int n = n_legs;
    tn::Step st;
    st.kind = 1;
    st.n = n;
    st.d.assign(leg_dim, leg_dim + n);
    st.D.assign(n, 1);
    for (int k = 0; k < n; ++k) {
      if (st.d[k] < 1) fail(TN_ERR_INVALID, "leg dim < 1");
      if (k < n - 1) {
        st.D[k] = bond_dim[k];
        if (st.D[k] < 1 || st.D[k] > (1 << 16)) fail(TN_ERR_INVALID, "bond dim out of range");
      }
    }
    st.site.resize(n);
    for (int k = 0; k < n; ++k) {
      tn::SiteOp o{};
      o.a = (k == 0) ? 1 : st.D[k - 1];
      o.b = st.D[k];
      o.dp = o.dhl = o.dhr = 1;
      o.de = st.d[k];
      st.site[k] = o;
    }
    st.r.assign(n - 1, 0);
    st.r[0] = st.d[0];
    for (int k = 1; k <= n - 2; ++k) {
      double beyond = 1;
      for (int j = k + 1; j < n; ++j) beyond *= st.d[j];
      const int ck_ = chi_per_edge ? chi_per_edge[k] : chi;
      if (ck_ < 1) fail(TN_ERR_INVALID, "chi_per_edge entries must be >= 1");
      double r = std::min<double>(ck_, double(st.r[k - 1]) * st.d[k]);
      r = std::min<double>(r, st.D[k]);
      r = std::min<double>(r, beyond);
      st.r[k] = int(r);
    }
    st.y_off.assign(n, 0);
    long long off = 0;
    for (int k = 0; k < n; ++k) {
      st.y_off[k] = off;
      off += (long long)st.site[k].a * st.d[k] * st.D[k];
    }
    st.y_total = off;
    st.s_off.assign(n, 0);
    st.s_size.assign(n, 0);
    off = 0;
    for (int k = 0; k < n; ++k) {
      const long long left = (k == 0) ? 1 : st.r[k - 1];
      const long long right = (k == n - 1) ? 1 : st.r[k];
      st.s_off[k] = off;
      st.s_size[k] = left * st.d[k] * right;
      off += st.s_size[k];
    }
    st.s_total = off;
    st.r_off.assign(n, 0);
    off = 0;
    for (int k = 1; k <= n - 1; ++k) {
      st.r_off[k] = off;
      off += (long long)st.D[k] * st.D[k];
    }
    st.r_total = off;
    tn_plan_t tmp;
    tmp.steps.push_back(st);
    const Dims dm = plan_dims(&tmp);
    // carve the static array: boundary sites, blocks, R_k, X, M, G, L, P, eigenvalues,
    // max-abs slots, log-scale and status per instance
    const long long B = n_inst;
    const size_t dbl = sizeof(double);
    const size_t parts[] = {dbl * size_t(dm.maxS * B),   dbl * size_t(dm.maxY * B),
                            dbl * size_t(dm.maxR * B),   dbl * size_t(dm.maxX * B),
                            dbl * size_t(dm.maxM * B),   dbl * size_t(dm.maxM * B),
                            dbl * size_t(dm.maxL * B),   dbl * size_t(dm.maxP * B),
                            dbl * size_t(dm.maxLam * B), sizeof(unsigned long long) * size_t(dm.maxN * B),
                            dbl * size_t(B),             sizeof(int) * size_t(B)};
    size_t offs[12], need = 0;
    for (int i = 0; i < 12; ++i) {
      offs[i] = need;
      need += align256(parts[i]);
    }
    if (need > TN_NOALLOC_SCRATCH_BYTES)
      fail(TN_ERR_INVALID, "problem needs " + std::to_string(need) +
                               " bytes of workspace; the static workspace holds " +
                               std::to_string(size_t(TN_NOALLOC_SCRATCH_BYTES)));
    int dev = 0;
    ck(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) fail(TN_ERR_INVALID, "device ordinal out of range");
    void* base_v = nullptr;
    {
      std::lock_guard<std::mutex> lock(g_noalloc_mu);
      if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        ck(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress");
        ck(tn::eigh_configure(), "eigh configure");
        g_noalloc_addr[dev] = p;
      }
      base_v = g_noalloc_addr[dev];
    }
    char* base = static_cast<char*>(base_v);
    Ws w{};
    w.sS = dm.maxS; w.sY = dm.maxY; w.sR = dm.maxR; w.sX = dm.maxX; w.sM = dm.maxM;
    w.sL = dm.maxL; w.sP = dm.maxP; w.sLam = dm.maxLam; w.sAmax = dm.maxN; w.sInv = 0;
    w.S0 = nullptr;
    w.inv = nullptr;
    w.S1 = reinterpret_cast<double*>(base + offs[0]);
    w.Y = reinterpret_cast<double*>(base + offs[1]);
    w.R = reinterpret_cast<double*>(base + offs[2]);
    w.X = reinterpret_cast<double*>(base + offs[3]);
    w.M = reinterpret_cast<double*>(base + offs[4]);
    w.G = reinterpret_cast<double*>(base + offs[5]);
    w.L = reinterpret_cast<double*>(base + offs[6]);
    w.P = reinterpret_cast<double*>(base + offs[7]);
    w.lam = reinterpret_cast<double*>(base + offs[8]);
    w.amax = reinterpret_cast<unsigned long long*>(base + offs[9]);
    // a ctx that owns no device memory, pointing at the static workspace
    tn_ctx local;
    local.device = dev;
    local.logscale = reinterpret_cast<double*>(base + offs[10]);
    local.status = reinterpret_cast<int*>(base + offs[11]);
    cudaStream_t strm = static_cast<cudaStream_t>(stream);
    // the array keeps the previous call's contents: reset what starts at zero
    ck(cudaMemsetAsync(local.logscale, 0, dbl * size_t(B), strm), "memset");
    ck(cudaMemsetAsync(local.status, 0, sizeof(int) * size_t(B), strm), "memset");
    for (int i = 0; i < n_inst; ++i)
      ck(cudaMemcpyAsync(w.Y + w.sY * i, blocks_dev[i], dbl * st.y_total,
                         cudaMemcpyDeviceToDevice, strm),
         "copy blocks");
    dm_pass(&local, st, w, w.S1, n_inst, TN_PREC_FP64, strm);
    for (int i = 0; i < n_inst; ++i)
      ck(cudaMemcpyAsync(tree_dev[i], w.S1 + w.sS * i + st.s_off[1],
                         dbl * (st.s_total - st.s_size[0]), cudaMemcpyDeviceToDevice, strm),
         "copy tree");
    ck(cudaMemcpyAsync(lognorm_dev, local.logscale, dbl * size_t(B), cudaMemcpyDeviceToDevice,
                       strm),
       "copy lognorm");
    ck(cudaMemcpyAsync(status_dev, local.status, sizeof(int) * size_t(B),
                       cudaMemcpyDeviceToDevice, strm),
       "copy status");
    for (int k = 0; k < n - 1; ++k) ranks_host[k] = st.r[k];
  });
}

extern "C" tn_status tn_autotune(tn_ctx_t* c, const tn_plan_t* const* plans, int32_t n_inst,
                                 const double* const* sites_dev, int32_t precision,
                                 const char* cache_path) {
  if (!c) {
    tn::set_error("tn_autotune: ctx is NULL");
    return TN_ERR_INVALID;
  }
  return guarded(c, "tn_autotune", [&] {
    if (!plans || !sites_dev || n_inst < 1) fail(TN_ERR_INVALID, "plans/sites NULL or n_inst < 1");
    for (int i = 0; i < n_inst; ++i)
      if (!plans[i] || !sites_dev[i]) fail(TN_ERR_INVALID, "NULL plan or site buffer");
    if (precision == TN_PREC_FP64) return;  // no tensor-core contraction to tune
    if (precision != TN_PREC_TF32 && precision != TN_PREC_TF32_FAST &&
        precision != TN_PREC_TF32_GRAM)
      fail(TN_ERR_UNSUPPORTED, "precision mode not implemented in this build");
    if (!c->tc_ready) fail(TN_ERR_UNSUPPORTED, "tcgen05 path unavailable on this device");
    ck(cudaSetDevice(c->device), "cudaSetDevice");
    cudaDeviceProp prop{};
    ck(cudaGetDeviceProperties(&prop, c->device), "cudaGetDeviceProperties");
    const std::string dev = prop.name;
    // a cache written for this device replaces the table
    if (cache_path) {
      if (FILE* f = std::fopen(cache_path, "r")) {
        std::map<std::array<int, 5>, std::array<int, 3>> t;
        char line[512];
        bool same_dev = false;
        while (std::fgets(line, sizeof line, f)) {
          if (std::strstr(line, "\"device\"") && std::strstr(line, dev.c_str())) same_dev = true;
          int M, N, K, sp, bt, bn, kb, ns;
          if (std::sscanf(line,
                          " {\"M\": %d, \"N\": %d, \"K\": %d, \"split\": %d, \"batch\": %d, "
                          "\"BN\": %d, \"budget_kb\": %d, \"ns\": %d}",
                          &M, &N, &K, &sp, &bt, &bn, &kb, &ns) == 8)
            t[{M, N, K, sp, bt}] = {bn, kb, ns};
        }
        std::fclose(f);
        if (same_dev && !t.empty()) {
          c->tune = std::move(t);
          return;
        }
      }
    }
    cudaStream_t strm = nullptr;
    c->tuning = true;
    try {
      run_batch(c, plans, n_inst, sites_dev, precision, false, strm, true);
      ck(cudaStreamSynchronize(strm), "cudaStreamSynchronize");
    } catch (...) {
      c->tuning = false;
      throw;
    }
    c->tuning = false;
    c->pending = false;
    if (cache_path) {
      FILE* f = std::fopen(cache_path, "w");
      if (!f) fail(TN_ERR_INVALID, std::string("cannot write ") + cache_path);
      std::fprintf(f, "{\"format\": \"tn_dmtree tcgen05 tiles v1\",\n \"device\": \"%s\",\n \"entries\": [\n",
                   dev.c_str());
      size_t i = 0;
      for (const auto& kv : c->tune) {
        std::fprintf(f,
                     "  {\"M\": %d, \"N\": %d, \"K\": %d, \"split\": %d, \"batch\": %d, \"BN\": %d, "
                     "\"budget_kb\": %d, \"ns\": %d}%s\n",
                     kv.first[0], kv.first[1], kv.first[2], kv.first[3], kv.first[4],
                     kv.second[0], kv.second[1], kv.second[2], (++i < c->tune.size()) ? "," : "");
      }
      std::fprintf(f, " ]}\n");
      std::fclose(f);
    }
  });
}

extern "C" tn_status tn_autotune_entries(const tn_ctx_t* c, int32_t* n_entries) {
  if (!c || !n_entries) {
    tn::set_error("tn_autotune_entries: NULL argument");
    return TN_ERR_INVALID;
  }
  *n_entries = int32_t(c->tune.size());
  return TN_OK;
}

// ---------------------------------------------------------------- graphs
struct tn_batch_graph {
  tn_ctx* own = nullptr;  // a private ctx: its workspace belongs to the graph
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int n = 0;
};

extern "C" tn_status tn_batch_graph_capture(tn_ctx_t* c, const tn_plan_t* const* plans, int32_t n_inst,
                                      const double* const* sites_dev, int32_t precision,
                                      tn_batch_graph_t** out) {
  if (!c || !out) {
    tn::set_error("tn_batch_graph_capture: ctx or out is NULL");
    return TN_ERR_INVALID;
  }
  *out = nullptr;
  tn_batch_graph* g = new (std::nothrow) tn_batch_graph();
  if (!g) {
    tn::set_error("tn_batch_graph_capture: host allocation failed");
    return TN_ERR_OOM;
  }
  cudaStream_t cap = nullptr;
  bool capturing = false;
  tn_status s = guarded(c, "tn_batch_graph_capture", [&] {
    if (!plans || !sites_dev || n_inst < 1) fail(TN_ERR_INVALID, "plans/sites NULL or n_inst < 1");
    for (int i = 0; i < n_inst; ++i)
      if (!plans[i] || !sites_dev[i]) fail(TN_ERR_INVALID, "NULL plan or site buffer");
    if (precision != TN_PREC_FP64 && precision != TN_PREC_TF32 &&
        precision != TN_PREC_TF32_FAST && precision != TN_PREC_TF32_GRAM)
      fail(TN_ERR_UNSUPPORTED, "precision mode not implemented in this build");
    const tn_status cs = tn_ctx_create(c->device, &g->own);
    if (cs != TN_OK) fail(cs, tn::get_error());
    if (precision != TN_PREC_FP64 && !g->own->tc_ready)
      fail(TN_ERR_UNSUPPORTED, "tcgen05 path unavailable on this device");
    g->own->eig_rounds = c->eig_rounds;
    g->own->tune = c->tune;
    g->own->grouped = c->grouped;
    g->own->value_comp = c->value_comp;
    g->n = n_inst;
    ck(cudaDeviceSynchronize(), "cudaDeviceSynchronize");  // site buffers ready for cap
    ck(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "cudaStreamCreate");
    // one eager run sizes the workspace and places the tables
    run_batch(g->own, plans, n_inst, sites_dev, precision, false, cap, true);
    ck(cudaStreamSynchronize(cap), "cudaStreamSynchronize");
    ck(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
    capturing = true;
    run_batch(g->own, plans, n_inst, sites_dev, precision, false, cap, false);
    capturing = false;
    ck(cudaStreamEndCapture(cap, &g->graph), "cudaStreamEndCapture");
    ck(cudaGraphInstantiate(&g->exec, g->graph, 0), "cudaGraphInstantiate");
    g->own->pending = false;
  });
  if (capturing && cap) {
    cudaGraph_t junk = nullptr;
    cudaStreamEndCapture(cap, &junk);
    if (junk) cudaGraphDestroy(junk);
    cudaGetLastError();
  }
  if (cap) cudaStreamDestroy(cap);
  if (s != TN_OK) {
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    if (g->own) tn_ctx_destroy(g->own);
    delete g;
    return s;
  }
  *out = g;
  return TN_OK;
}

extern "C" tn_status tn_batch_graph_launch(tn_batch_graph_t* g, void* stream) {
  if (!g || !g->exec) {
    tn::set_error("tn_batch_graph_launch: graph is NULL");
    return TN_ERR_INVALID;
  }
  return guarded(g->own, "tn_batch_graph_launch", [&] {
    ck(cudaSetDevice(g->own->device), "cudaSetDevice");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    ck(cudaGraphLaunch(g->exec, st), "cudaGraphLaunch");
    g->own->stream = st;
    g->own->last_batch = g->n;
    g->own->pending = true;
  });
}

extern "C" tn_status tn_batch_graph_logz(tn_batch_graph_t* g, double* logz_host, int32_t* status_host,
                                   int32_t n_inst) {
  if (!g) {
    tn::set_error("tn_batch_graph_logz: graph is NULL");
    return TN_ERR_INVALID;
  }
  return tn_logz(g->own, logz_host, status_host, n_inst);
}

extern "C" tn_status tn_batch_graph_destroy(tn_batch_graph_t* g) {
  if (!g) return TN_OK;
  if (g->own) {
    cudaSetDevice(g->own->device);
    cudaDeviceSynchronize();
  }
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  if (g->own) tn_ctx_destroy(g->own);
  delete g;
  return TN_OK;
}

extern "C" tn_status tn_ctx_set_option(tn_ctx_t* c, int32_t option, int64_t value) {
  if (!c) {
    tn::set_error("tn_ctx_set_option: ctx is NULL");
    return TN_ERR_INVALID;
  }
  return guarded(c, "tn_ctx_set_option", [&] {
    if (option == TN_OPT_EIG_ROUNDS) {
      if (value < 1 || value > 16) fail(TN_ERR_INVALID, "TN_OPT_EIG_ROUNDS must be 1 .. 16");
      c->eig_rounds = int(value);
    } else if (option == TN_OPT_WAIT_PROBE) {
      c->wait_probe = value != 0;
    } else if (option == TN_OPT_VALUE_PATH) {
      if (value != 0 && value != 1) fail(TN_ERR_INVALID, "TN_OPT_VALUE_PATH must be 0 or 1");
      c->value_comp = value != 0;
    } else if (option == TN_OPT_GROUPED) {
      if (value != 0 && value != 1) fail(TN_ERR_INVALID, "TN_OPT_GROUPED must be 0 or 1");
      c->grouped = value != 0;
    } else {
      fail(TN_ERR_INVALID, "unknown option");
    }
  });
}

extern "C" tn_status tn_ctx_set_profiling(tn_ctx_t* c, int32_t on) {
  if (!c) {
    tn::set_error("tn_ctx_set_profiling: ctx is NULL");
    return TN_ERR_INVALID;
  }
  c->prof = (on != 0);
  return TN_OK;
}

extern "C" tn_status tn_ctx_profile(tn_ctx_t* c, double* ms_host, int64_t* launches_host,
                                    int32_t n_classes) {
  if (!c) {
    tn::set_error("tn_ctx_profile: ctx is NULL");
    return TN_ERR_INVALID;
  }
  return guarded(c, "tn_ctx_profile", [&] {
    if (n_classes < 0 || n_classes > TN_KC_COUNT || !launches_host)
      fail(TN_ERR_INVALID, "invalid argument");
    ck(cudaSetDevice(c->device), "cudaSetDevice");
    ck(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    double ms[TN_KC_COUNT] = {};
    for (const auto& r : c->recs) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) ms[r.cls] += t;
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
    cudaGetLastError();
    c->recs.clear();
    for (int k = 0; k < n_classes; ++k) {
      launches_host[k] = c->launches[k];
      if (ms_host) ms_host[k] = ms[k];
    }
    for (int k = 0; k < TN_KC_COUNT; ++k) c->launches[k] = 0;
  });
}

extern "C" const char* tn_last_error(const tn_ctx_t* c) {
  if (c && !c->err.empty()) return c->err.c_str();
  return tn::get_error();
}
