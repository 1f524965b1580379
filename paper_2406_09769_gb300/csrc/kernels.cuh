// Kernel launch interfaces of the density-matrix tree approximation.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace tn {

// One tree vertex's block fusion (device copy of SiteOp plus buffer offsets).
struct FuseSite {
  int32_t vertex, a, dp, b, dhl, dhr, de, pad;
  int64_t t_off, sp, shl, shr, se;
  int64_t y_off, s_off;
};

// Batched row-major GEMM  C_i = alpha_i * op(A_i) op(B_i), i = 0..batch-1,
// X_i = X + i * sX.  alpha_i = 1 / amax_in[i * s_amax_in] when amax_in is set
// (the running max-abs of a memoised density matrix), else 1.  When amax_out is
// set, max |C_i| is folded into amax_out[i * s_amax_out] (bits of a
// non-negative double, atomicMax; zero it first).
struct GemmArgs {
  const double* A; long long sA; int lda;
  const double* B; long long sB; int ldb;
  double* C; long long sC; int ldc;
  int M, N, K, batch;
  const unsigned long long* amax_in; long long s_amax_in;
  unsigned long long* amax_out; long long s_amax_out;
};

cudaError_t launch_dgemm(bool ta, bool tb, const GemmArgs& g, cudaStream_t st);

// Batched tcgen05 contraction C_i = alpha_i * A_i B_i^T with FP32 operands,
// TF32 tensor-core products and FP32 accumulation (K-major A: M x K, B: N x K).
// lda, ldb, sA, sB must be multiples of 4 elements and A, B 16-byte aligned.
// C (row-major, ldc) and/or Ct (= C^T, row-major, ldct) may be NULL.  alpha_i =
// 1 / amax_in[i * s_amax_in] (float bits) when amax_in is set.  amax_out gets
// max |C_i| (float bits, atomicMax; zero it first).  split = 1 adds the two
// cross terms of a hi/lo TF32 split (compensated, ~FP32 accurate).  *err is
// set to 1 if a bounded wait expired.
struct TcGemmArgs {
  const float* A; long long sA; int lda;
  const float* B; long long sB; int ldb;
  float* C; long long sC; int ldc;
  float* Ct; long long sCt; int ldct;
  int M, N, K, batch;
  const unsigned int* amax_in; long long s_amax_in;
  unsigned int* amax_out; long long s_amax_out;
  int split;
  int ct_cols;   // C^T store groups columns n = q * ct_cols + c into Ct[c][m * (N / ct_cols) + q]
  int* err;
  const int* poll;  // if set: a bounded wait on *poll != 0 first (expiry -> *err = 1)
  int bn;           // tile width (multiple of 16, <= 256), 0: round_up(N, 16) capped at 256
  int budget_kb;    // shared-memory budget of the K-chunk ring, 0: 104 KB (two CTAs per SM)
};
cudaError_t tc_gemm_configure();
cudaError_t launch_sgemm_nt(const TcGemmArgs& g, cudaStream_t st);
// FP32 FFMA (round to nearest) tiled GEMM of the same form: the value path;
// compensated: Kahan accumulation (about FP64-accumulation accuracy).
cudaError_t launch_sgemm_ffma(const TcGemmArgs& g, bool compensated, cudaStream_t st);
cudaError_t launch_tc_gemm(const TcGemmArgs& g, cudaStream_t st);
size_t tc_gemm_smem_bytes(int BN, int split, int K, int* stages_out, int budget_kb = 104);

cudaError_t launch_site_norm(const double* const* tens, const int64_t* off, const int64_t* len,
                             int nv, int batch, double* inv_norm, double* logscale, int* status,
                             cudaStream_t st);

cudaError_t launch_fuse(const FuseSite* sites, int n, int max_elems, const double* const* tens,
                        const double* inv_norm, int nv, const double* S, long long sS,
                        int trivial, double* Y, long long sY, int batch, cudaStream_t st);

cudaError_t launch_fill_env_root(double* R, long long sR, unsigned long long* amax,
                                 long long s_amax, int batch, cudaStream_t st);

cudaError_t launch_root(const double* P, long long sP, const double* Y, long long sY, int r, int D,
                        int d, double* S_root, double* S_first, int d0, long long sS,
                        double* logscale, int* status, int batch, cudaStream_t st);

cudaError_t launch_close(const double* Y, long long sY, const int64_t* y_off, const int32_t* D,
                         int n, int maxD, const double* logscale, double* logz, int* status,
                         int batch, cudaStream_t st);

// Batched top-r symmetric eigensolver: U_i (n x r, row-major, descending
// eigenvalues, columns signed so the largest-|.| entry is positive) and
// lam_i[0..nlam) (descending).  One CTA per matrix.
template <typename T>
cudaError_t launch_eigh_top(const T* L, long long sL, T* U, long long sU, T* Ut, long long sUt,
                            double* lam, long long slam, int n, int r, int nlam, int* status,
                            int batch, cudaStream_t st);

// FP32-storage kernels of the mixed-precision path (see kernels_f32.cu).
// bond2: all sites but at most two (a row's end sites) have dp = dhl = dhr =
// de = 2 and even Y offsets; max_a, max_b: largest a and b over the sites.
cudaError_t launch_fuse_f32(const FuseSite* sites, int n, int max_elems, int max_dl, int max_j,
                            int max_t, int max_a, int max_b, int bond2,
                            const double* const* tens,
                            const double* inv_norm, int nv, const float* S, long long sS,
                            int trivial, float* Y, long long sY, float* Yt, const int64_t* yt_off,
                            int batch, cudaStream_t st);
cudaError_t launch_fill_env_root_f32(float* R, long long sR, unsigned int* amax, long long s_amax,
                                     int batch, cudaStream_t st);
cudaError_t launch_root_f32(const float* P, long long sP, int ldp, const float* Y, long long sY,
                            int r, int D, int d, float* S_root, float* S_first, int d0,
                            long long sS, double* logscale, int* status, int batch,
                            cudaStream_t st);
cudaError_t launch_close_f32(const float* Y, long long sY, const int64_t* y_off, const int32_t* D,
                             int n, int maxD, const double* logscale, double* logz, int* status,
                             int batch, cudaStream_t st);
// Segment conversions between the caller's FP64 buffers and FP32 workspace
// (one pass on explicit blocks in the mixed precision, tn_embed_tree).
struct CvtSeg {
  int64_t src_off, dst_off;
  int32_t rows, cols;
};
cudaError_t launch_convert_segments_d2f(const double* const* src_tab, float* dst_base,
                                        long long s_dst, float* dst_t, const CvtSeg* segs,
                                        int nseg, int max_elems, int batch, cudaStream_t st);
cudaError_t launch_convert_segments_f2d(const float* src_base, long long s_src,
                                        double* const* dst_tab, const CvtSeg* segs, int nseg,
                                        int max_elems, int batch, cudaStream_t st);
// ---- learned per-edge rank allocation (learned.cu)
constexpr int kRankFeatures = 22;
constexpr int kRankHidden = 64;
struct RankArgs {
  const double* lam; long long slam;  // descending eigenvalues of L_v, A of them per instance
  int A, rk, dk;                      // dim A_v, structural rank of the chi_max plan, d_v
  int v, nlegs, pass, npass;          // tree vertex, legs, DM pass index, DM passes
  const void* model;                  // BF16 MLP parameters, or NULL: keep rk, record only
  int budget_total, edges_after, first;  // per-pass budget; later vertices; first vertex
  int chi_uniform;                    // rank of the uniform method the budget is taken from
  int reserve_after;                  // budget kept for later vertices: sum min(2, r_u)
  int* budget_rem;                    // per-instance running budget
  int* prev_chi;                      // per-instance rank kept at the previous vertex
  double* acc;                        // per-instance summed discarded share (or NULL)
  int* rec_chi; float* rec_feat; double* rec_spec; long long rec_off;  // optional records
  int fixed_chi;                      // no model: keep min(fixed_chi, r_v) (0: r_v)
};
int rank_model_params();
template <typename T>
cudaError_t launch_rank_select(const RankArgs& g, T* U, long long sU, T* Ut, long long sUt,
                               int batch, cudaStream_t st);
cudaError_t launch_mlp_grad(const float* X, const float* tgt, const int* idx, int n, float scale,
                            const float* w, float* grad, float* loss, cudaStream_t st);
cudaError_t launch_adam(float* w, float* grad, float* m, float* v, int np, float lr, float b1,
                        float b2, float eps, int t, cudaStream_t st);
cudaError_t launch_to_bf16(const float* w, void* out, int np, cudaStream_t st);
cudaError_t launch_water_fill(const double* spec, const int* cap, const int* pass_start,
                              int chi_u, int n_pass, int B, int* chi_out, float* feat,
                              cudaStream_t st);
int water_fill_max_edges();
// Per instance: keep ln Z / status of the run with the smaller summed discarded
// share (learned run: logz, status in place; uniform run: logz_u, status_u);
// used[i] = 1 where the learned run is kept.
cudaError_t launch_judge_select(const double* acc_l, const double* acc_u, const double* logz_u,
                                const int* status_u, double* logz, int* status, int* used,
                                int n, cudaStream_t st);
cudaError_t launch_iota(int* x, int n, cudaStream_t st);

// Factored density matrices (svd.cu).  launch_chol_env: every memoised
// environment R_k (k = k0 .. k0 + nk - 1, n = D[k] <= 128, at R + i sR +
// r_off[k], scaled by 1 / amax[i s_amax + k] as float bits) is replaced in
// place by C^T (row-major) with R_k / amax = C C^T, C lower triangular.
// launch_svd_left: the r (<= 64) leading left singular vectors of K_i (m x n,
// row-major, m, n <= 128) into U (m x r) and Ut (r x m, may be NULL), signed
// so the largest-|.| entry is positive, and sigma_t^2 for t < nlam into lam.
// ---- grouped launches: one launch over problems of different buckets (plans)
// and shapes; every problem carries its own pointers.
// Range guard (a diagnostic mode of the grouped executor): the sorted device
// allocations [lo[i], hi[i]) every global access must fall in.  A kernel whose
// descriptor carries a guard checks each global access before making it; the
// first one outside every allocation is recorded in rec (tag + 1, linear
// block index, address, bytes) and skipped.
struct GuardTab {
  const unsigned long long* lo;
  const unsigned long long* hi;
  unsigned long long* rec;
  int n, pad;
};
#ifdef __CUDACC__
__device__ __forceinline__ bool guard_ok(const GuardTab* g, const void* p, long long bytes,
                                         int tag) {
  if (!g) return true;
  const unsigned long long a = reinterpret_cast<unsigned long long>(p);
  int lo = 0, hi = g->n - 1, f = -1;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    if (g->lo[mid] <= a) {
      f = mid;
      lo = mid + 1;
    } else {
      hi = mid - 1;
    }
  }
  if (f >= 0 && bytes >= 0 && a + (unsigned long long)bytes <= g->hi[f]) return true;
  if (atomicCAS(g->rec, 0ull, (unsigned long long)tag + 1ull) == 0ull) {
    g->rec[1] = blockIdx.x + (unsigned long long)gridDim.x *
                                 (blockIdx.y + (unsigned long long)gridDim.y * blockIdx.z);
    g->rec[2] = a;
    g->rec[3] = (unsigned long long)bytes;
  }
  return false;
}
// A note of the guard mode: records (tag, block, v0, v1) if nothing was
// recorded before.
__device__ __forceinline__ void guard_note(const GuardTab* g, int tag, unsigned long long v0,
                                           unsigned long long v1) {
  if (!g) return;
  if (atomicCAS(g->rec, 0ull, (unsigned long long)tag + 1ull) == 0ull) {
    g->rec[1] = blockIdx.x + (unsigned long long)gridDim.x *
                                 (blockIdx.y + (unsigned long long)gridDim.y * blockIdx.z);
    g->rec[2] = v0;
    g->rec[3] = v1;
  }
}
// An index check of the guard mode: false (and recorded, value in place of
// the address) unless 0 <= v < lim.
__device__ __forceinline__ bool guard_idx(const GuardTab* g, long long v, long long lim, int tag) {
  if (!g || (v >= 0 && v < lim)) return true;
  if (atomicCAS(g->rec, 0ull, (unsigned long long)tag + 1ull) == 0ull) {
    g->rec[1] = blockIdx.x + (unsigned long long)gridDim.x *
                                 (blockIdx.y + (unsigned long long)gridDim.y * blockIdx.z);
    g->rec[2] = (unsigned long long)v;
    g->rec[3] = (unsigned long long)lim;
  }
  return false;
}
#endif
struct SvdDesc {
  const float* K; float* U; float* Ut; double* lam; int* status;
  int m, n, r, nlam;
  const GuardTab* guard;
};
struct CholDesc {
  float* R; const unsigned int* amax; int n, pad;
  const GuardTab* guard;
};
// C = alpha A B^T (A: M x K, B: N x K, K-major), alpha = 1 / *amax_in if set;
// Ct (optional): columns grouped as in TcGemmArgs::ct_cols; max|C| folded
// into *amax_out if set.
struct GemmDesc {
  const float* A; const float* B; float* C; float* Ct;
  const unsigned int* amax_in; unsigned int* amax_out;
  int M, N, K, lda, ldb, ldc, ldct, ct_cols;
  const GuardTab* guard;
};
struct RootDesc {
  const float* P; const float* Y; float* S_root; float* S_first;
  double* logscale; int* status;
  int ldp, r, D, d, d0, pad;
  const GuardTab* guard;
};
// Start of a pass: amax[0 .. n-2] = 0, R_{n-1} = [1] at R, amax[n-1] = 1.
struct EnvRootDesc {
  float* R; unsigned int* amax; int n, pad;
  const GuardTab* guard;
};
cudaError_t launch_svd_left_grouped(const SvdDesc* desc, int n_prob, int max_m, int max_n,
                                    int max_r, bool guarded, cudaStream_t st, int rounds = 9);
cudaError_t launch_chol_grouped(const CholDesc* desc, int n_prob, bool guarded, cudaStream_t st);
cudaError_t launch_gemm_grouped(const GemmDesc* desc, int n_prob, int max_M, int max_N,
                                bool compensated, bool guarded, cudaStream_t st);
cudaError_t launch_root_grouped(const RootDesc* desc, int n_prob, int max_rd, bool guarded,
                                cudaStream_t st);
cudaError_t launch_env_root_grouped(const EnvRootDesc* desc, int n_prob, cudaStream_t st);
// FP32 leading eigenvectors of L (n x n, n <= 128, r <= 64) per problem.
struct EighDesc {
  const float* L; float* U; float* Ut; double* lam; int* status;
  int n, r, nlam, pad;
  const GuardTab* guard;
};
cudaError_t launch_eigh_grouped(const EighDesc* desc, int n_prob, int max_n, int max_r,
                                bool guarded, cudaStream_t st);
cudaError_t launch_chol_env(float* R, long long sR, const int64_t* r_off, const int32_t* D,
                            int maxD, const unsigned int* amax, long long s_amax, int k0, int nk,
                            int batch, cudaStream_t st);
// rounds: multisection rounds after the shared grid round (1 .. 16; 9
// resolve every interval to ~4e-9 ||T||); an interval left wider than 128
// eps ||T|| marks the instance TN_ERR_EIG_NOCONV.
cudaError_t launch_svd_left(const float* K, long long sK, int m, int n, float* U, long long sU,
                            float* Ut, long long sUt, double* lam, long long slam, int r,
                            int nlam, int* status, int batch, cudaStream_t st, int rounds = 9);
bool svd_left_supported(int m, int n, int r);
size_t svd_left_smem_bytes(int m, int n, int r);
cudaError_t svd_configure();

// Blocks of general plans (gather.cu).  One op of a chain position's program
// (device copy of GOpH with resolved offsets): out[e] = sum over the summed
// slots of the product of its operands, e decoded row-major into the output
// slots (a slot listed twice must take equal digits, else 0).  Output: the
// block (y_off into Y and, if Yt is set, its transpose (dkDr x Dl) into Yt)
// or scratch at dst_off.
struct GOp {
  int64_t dst_off, n_elems;
  int32_t to_block, Dl, dkDr, ns, nout, nsum, nt, t_first, code_off, pad;
};
// An operand: src 0 = raw site tensor (tens[i] + base, times inv[vertex]),
// 1 = MPS site of the previous step (S + base), 2 = scratch (scr + base).
struct GTen {
  int64_t base;
  int32_t src, vertex, nleg, leg_off;
};
// Runs ops [a, b) of one level; pre: exclusive prefix of n_elems over all ops
// of the step (pre[i] .. pre[i+1] are op i's elements).
// Grouped gather (FP32 path): one problem = ops [a, b) of one bucket's step
// for one instance, with that instance's pointers.
struct GatherDesc {
  const GOp* ops; const GTen* ten; const int32_t* code; const int64_t* pre;
  const double* raw; const double* inv; const float* S; double* scr; float* Y; float* Yt;
  int a, b;
  const GuardTab* guard;
};
cudaError_t launch_gather_grouped(const GatherDesc* desc, int n_prob, int64_t max_elems,
                                  bool guarded, cudaStream_t st);
template <typename TS, typename TY>
cudaError_t launch_gather(const GOp* ops, const GTen* ten, const int32_t* code, const int64_t* pre,
                          int a, int b, int64_t n_elems, const double* const* tens,
                          const double* inv, long long sInv, const TS* S, long long sS,
                          double* scr, long long sScr, TY* Y, long long sY, TY* Yt, int batch,
                          cudaStream_t st);

template <typename T>
size_t eigh_smem_bytes(int n, int r, int nlam);
template <typename T>
size_t eigh_smem_limit();
template <typename T>
size_t eigh_fast_smem_limit();
cudaError_t eigh_configure();

}  // namespace tn
