// Factored density matrices of the mixed-precision path.
//
// Algorithm density_matrix_alg (Sec. 5) keeps the leading eigenvectors of
// L_v = M_v R_v M_v^T, with R_v the memoised root-side density matrix of
// Eq. dm_cache.  Forming L_v in FP32 squares the conditioning of M_v: its
// rounding (~6e-8 of the largest eigenvalue) drowns every eigen-direction
// below that level, and a truncation that falls there picks a subspace that
// does not belong to the stored state.  This file never forms L_v:
//   1. k_chol_env: R_v = C_v C_v^T (FP32 Cholesky with diagonal pivoting,
//      one CTA per R_v, every R_v of a pass in one launch).  The largest
//      remaining diagonal entry is eliminated first and rows are not swapped
//      (C = P L in the original row order); the factorisation stops once the
//      remaining diagonal is below eps^2 of the first pivot, so a
//      rank-deficient environment needs no shift.  Without pivoting, a
//      rounding-level pivot met before the end divides the rest of its
//      column by its square root and corrupts every later column;
//   2. K_v = M_v C_v on the tensor cores (compensated TF32, elsewhere);
//   3. k_svd_left: the leading left singular vectors of K_v, which are the
//      leading eigenvectors of L_v = K_v K_v^T, and sigma^2 as its
//      eigenvalues.  Backward error eps ||K_v|| on K_v is eps^2 ||L_v|| on
//      the density matrix.
// The SVD follows the bisection-and-inverse-iteration route of Marques,
// Demmel and Vasconcelos (LAPACK xBDSVDX):
//   a. Golub-Kahan bidiagonalisation K = H B G^T by Householder reflectors
//      (Golub & Van Loan, Matrix Computations, Sec. 5.4.8), K in register
//      tiles, left reflectors kept, right reflectors dropped;
//   b. the r largest eigenvalues of the Golub-Kahan tridiagonal T_GK (zero
//      diagonal, off-diagonals d_0, e_0, d_1, e_1, ...; eigenvalues
//      +-sigma_i) by Sturm-sequence multisection;
//   c. eigenvectors of T_GK by inverse iteration with partial pivoting; the
//      entries at odd positions are the left singular vector of B;
//   d. modified Gram-Schmidt (two passes), back-transformation
//      U = H_0 ... H_{p-1} [u; 0],
//      and each column signed so that its largest-|.| entry (first on ties)
//      is positive.
// Every loop has a fixed iteration bound; nothing waits on other blocks.
#include <cuda_runtime.h>

#include <cfloat>
#include <cmath>
#include <cstdint>

#include "kernels.cuh"
#include "tn_dmtree.h"

namespace tn {

namespace {

constexpr int kThreads = 256;
constexpr int kNmax = 128;   // largest m, n of K
constexpr int kRmax = 64;    // most singular vectors kept
constexpr int kQ = 32;       // rows of a vector held by one thread of a quad

__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float quad_sum(float v) {
  const unsigned qm = 0xFu << (threadIdx.x & 28);
  v += __shfl_xor_sync(qm, v, 1);
  v += __shfl_xor_sync(qm, v, 2);
  return v;
}

// ------------------------------------------------------------- Cholesky
// One CTA per (instance, tree vertex k): A = (R_k + R_k^T) / (2 max|R_k|),
// right-looking unblocked Cholesky A = C C^T in FP32 with the matrix in
// registers, thread (a = 2 warp + lane / 16, b = lane % 16) holding the 8 x 8
// tile A[8a .. 8a+7][8b .. 8b+7].  Step j: the owners of column j published
// it; every thread takes the pivot and its rows' and columns' entries of
// column j (A is kept symmetric, so row j equals column j), updates its tile
// A -= a_j a_j^T / pivot on rows and columns beyond j, and the owners of
// column j + 1 publish it: one barrier per step.  Row j of the output, C^T,
// is written straight from the published column.  A pivot that is not
// positive (round-off of a semi-definite R) leaves column j of C zero and the
// trailing block untouched.  Output in place of R_k: B[j][l] = C[l][j]
// (row-major, upper triangular), the K-major second operand of K = M C.
// kMode 0: strided batch; 1: grouped (CTA i factors problem desc[i]); 2: as 1
// with the range guard checked on every global access.
template <int kMode>
__global__ void __launch_bounds__(kThreads, 2) k_chol_env(float* __restrict__ R, long long sR,
                                                          const int64_t* __restrict__ r_off,
                                                          const int32_t* __restrict__ D,
                                                          const unsigned int* __restrict__ amax,
                                                          long long s_amax, int k0, int nk,
                                                          const CholDesc* __restrict__ desc) {
  __shared__ __align__(16) float Xc[128];
  __shared__ float dg[128];
  __shared__ int dn[128];
  int n;
  float* Rg;
  float am;
  const GuardTab* gd = nullptr;
  if (kMode) {  // grouped launch: CTA i factors problem desc[i]
    const CholDesc d = desc[blockIdx.x];
    gd = kMode == 2 ? d.guard : nullptr;
    n = d.n;
    Rg = d.R;
    am = guard_ok(gd, d.amax, 4, 0x401) ? __uint_as_float(*d.amax) : 1.f;
  } else {
    const int b = blockIdx.x / nk;
    const int k = k0 + blockIdx.x % nk;
    n = D[k];
    Rg = R + (long long)b * sR + r_off[k];
    am = __uint_as_float(amax[(long long)b * s_amax + k]);
  }
  const float sc = (am > 0.f && isfinite(am)) ? 0.5f / am : 0.5f;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ta = 2 * warp + (lane >> 4), tb = lane & 15;
  const int r0 = 8 * ta, c0 = 8 * tb;
  float t[8][8];
#pragma unroll
  for (int ii = 0; ii < 8; ++ii)
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
      const int i = r0 + ii, c = c0 + jj;
      t[ii][jj] = (i < n && c < n && guard_ok(gd, Rg + (long long)i * n + c, 4, 0x402) &&
                   guard_ok(gd, Rg + (long long)c * n + i, 4, 0x402))
                      ? (Rg[(long long)i * n + c] + Rg[(long long)c * n + i]) * sc
                      : 0.f;
    }
  if (tid < 128) dn[tid] = 0;
  __syncthreads();  // every load of R_k done before the first store of C^T
  float first = 0.f;
  for (int j = 0; j < n; ++j) {
    // the diagonal of the trailing matrix, eliminated rows excluded
    if (ta == tb)
#pragma unroll
      for (int ii = 0; ii < 8; ++ii) {
        const int i = r0 + ii;
        if (i < n) dg[i] = dn[i] ? -1.f : t[ii][ii];
      }
    __syncthreads();
    // pivot: the largest remaining diagonal entry (first index on ties),
    // found by every warp
    float pv = -1.f;
    int pi = n;
    for (int i = lane; i < n; i += 32) {
      const float x = dg[i];
      if (x > pv) { pv = x; pi = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float ov = __shfl_xor_sync(0xffffffffu, pv, o);
      const int oi = __shfl_xor_sync(0xffffffffu, pi, o);
      if (ov > pv || (ov == pv && oi < pi)) { pv = ov; pi = oi; }
    }
    if (j == 0) first = pv;
    // stop below eps^2 of the first pivot (or at a non-finite one): the
    // rounding of R_k (eps of its largest entry) then bounds every later
    // entry of C by O(sqrt(first pivot)).  Pivots between eps^2 and eps of
    // the first still carry environment directions that the truncation
    // needs; dropping them biases which subspace the next vertices keep.
    const bool ok = isfinite(pv) && pv > FLT_EPSILON * FLT_EPSILON * first && pv > 0.f;
    if (!ok) {
      for (long long q = (long long)j * n + tid; q < (long long)n * n; q += kThreads)
        if (guard_ok(gd, Rg + q, 4, 0x403)) Rg[q] = 0.f;
      break;
    }
    if (tb == (pi >> 3)) {
      switch (pi & 7) {
#define TN_CHOL_PUB(E) \
  case E: {            \
    _Pragma("unroll") for (int ii = 0; ii < 8; ++ii) Xc[r0 + ii] = t[ii][E]; \
  } break;
        TN_CHOL_PUB(0) TN_CHOL_PUB(1) TN_CHOL_PUB(2) TN_CHOL_PUB(3)
        TN_CHOL_PUB(4) TN_CHOL_PUB(5) TN_CHOL_PUB(6) TN_CHOL_PUB(7)
#undef TN_CHOL_PUB
      }
    }
    if (tid == 0) dn[pi] = 1;
    __syncthreads();
    const float ip = 1.f / pv;
    const float rs = rsqrtf(pv);
    // column j of C (row j of C^T): a_lp / sqrt(a_pp) on the rows not yet
    // eliminated, sqrt(a_pp) on the pivot row, 0 on eliminated rows (C = P L
    // in the original row order; C C^T = R_k / amax all the same)
    for (int l = tid; l < n; l += kThreads) {
      float v = 0.f;
      if (l == pi) v = pv * rs;
      else if (!dn[l]) v = Xc[l] * rs;
      if (guard_ok(gd, Rg + (long long)j * n + l, 4, 0x404)) Rg[(long long)j * n + l] = v;
    }
    // rank-1 update of the whole tile (eliminated rows and columns are never
    // read again)
    const float4 ra = *reinterpret_cast<const float4*>(Xc + r0);
    const float4 rb = *reinterpret_cast<const float4*>(Xc + r0 + 4);
    const float4 ca = *reinterpret_cast<const float4*>(Xc + c0);
    const float4 cb = *reinterpret_cast<const float4*>(Xc + c0 + 4);
    const float rv[8] = {ra.x, ra.y, ra.z, ra.w, rb.x, rb.y, rb.z, rb.w};
    const float cv[8] = {ca.x, ca.y, ca.z, ca.w, cb.x, cb.y, cb.z, cb.w};
    float cm[8];
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) cm[jj] = cv[jj] * ip;
#pragma unroll
    for (int ii = 0; ii < 8; ++ii) {
      const float2 nr = make_float2(-rv[ii], -rv[ii]);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float2 x = __ffma2_rn(nr, make_float2(cm[2 * q], cm[2 * q + 1]),
                                    make_float2(t[ii][2 * q], t[ii][2 * q + 1]));
        t[ii][2 * q] = x.x;
        t[ii][2 * q + 1] = x.y;
      }
    }
  }
}

// ---------------------------------------------------------------- SVD
// Bidiagonalisation layout: a 16 x 16 thread grid, thread (a = 2 warp + lane /
// 16, b = lane % 16) holds the 8 x 8 tile K[8a .. 8a+7][8b .. 8b+7] in
// registers (zero outside m x n).  Step k needs column k (left reflector) and
// row k (right reflector): their owners publish them to shared memory at the
// end of step k - 1.  Every warp forms the reflector scalars itself from the
// published vectors (same arithmetic, same values in each), so a step has two
// barriers: one after the per-warp column sums u^T K, one after the update.
//   column sums  w = tau K^T u : FMAs on the tile, the warp's two tile rows
//                combined by a shuffle, the eight warps' partials summed by
//                every reader from shared memory;
//   row sums     K v          : FMAs on the tile, summed over the sixteen
//                lanes of a tile row by a butterfly (bitwise the same in
//                every lane);
//   update       K -= u w^T + z v^T with z = tau' (K v - u (w . v)), all in
//                registers (u, z zero outside rows k+1 .. m-1, w, v outside
//                columns k+1 .. n-1, so the whole tile updates unmasked).
// Vectors phase: thread quad (column col = tid / 4, quarter qr = tid % 4)
// holds rows 32 qr .. 32 qr + 31 of its vector; shared vectors use padded
// rows (row c at c + 4 (c / 32)), so the quad's float4 reads hit disjoint bank
// groups.  Left reflector k is kept from row 4 floor(k / 4) to mr - 1 (mr = m
// rounded up to 4) in padded coordinates, back to back.
constexpr int kRld = 144;
__host__ __device__ __forceinline__ int rpad(int c) { return c + (c >> 5) * 4; }

__host__ __device__ inline int refl_len(int k, int m) {
  const int mr = (m + 3) & ~3;
  return rpad(mr) - rpad(k & ~3);
}

__host__ __device__ inline int refl_total(int m, int p) {
  int t = 0;
  for (int k = 0; k < p; ++k) t += refl_len(k, m);
  return t;
}

// floats after the reflectors and the Golub-Kahan vectors
constexpr int kSmallFloats = 256 + 256 + 1024 + 4 * 128 + 3 * 256 + 2 * kRld + 64 + 16 + 132 + 128;

// Sturm count of T_GK - x I (zero diagonal; eigenvalues below x).  The
// recurrence q_0 = -x, q_j = -x - g_{j-1}^2 / q_{j-1} is taken two entries
// at a time: with t = x q + g^2, the odd entry is q' = -t / q (only its sign
// is needed, and q' < 0 exactly when t and q have the same sign) and the next
// even entry is q'' = -x + g'^2 q / t, one division per pair.  Pivots below
// pivmin in magnitude count as -pivmin, as in the plain recurrence.
__device__ int sturm_gk(const float* e2, int N, float x, float pivmin) {
  float q = -x;
  if (fabsf(q) < pivmin) q = -pivmin;
  int c = (q < 0.f);
  int j = 1;
  for (; j + 1 < N; j += 2) {
    const float t = fmaf(x, q, e2[j - 1]);
    float qn;
    if (fabsf(t) < pivmin * fabsf(q)) {  // q' = -pivmin
      c += 1;
      qn = fmaf(e2[j], __fdividef(1.f, pivmin), -x);
    } else {
      c += ((t > 0.f) == (q > 0.f));
      qn = fmaf(e2[j], __fdividef(q, t), -x);
    }
    if (fabsf(qn) < pivmin) qn = -pivmin;
    c += (qn < 0.f);
    q = qn;
  }
  if (j < N) {  // a last odd entry
    const float t = fmaf(x, q, e2[j - 1]);
    c += (fabsf(t) < pivmin * fabsf(q)) ? 1 : ((t > 0.f) == (q > 0.f));
  }
  return c;
}

// Householder reflector for x = (alpha, tail) with s = |tail|^2: returns
// beta (the new leading entry), tau and the tail scale sc (u = (1, sc tail)).
// tau = 2 / (u^T u) = 2 / (1 + s sc^2) keeps H = I - tau u u^T orthogonal to
// working precision whatever the rounding of beta and sc.
__device__ __forceinline__ void house(float alpha, float s, float& beta, float& tau, float& sc) {
  if (s == 0.f) {
    beta = alpha; tau = 0.f; sc = 0.f;
    return;
  }
  const float nrm = sqrtf(fmaf(alpha, alpha, s));
  beta = (alpha >= 0.f) ? -nrm : nrm;
  sc = __fdividef(1.f, alpha - beta);
  tau = __fdividef(2.f, fmaf(s, sc * sc, 1.f));
}

// sum over the sixteen lanes of a half warp (butterfly: every lane gets the
// same bits)
__device__ __forceinline__ float half_sum(float v) {
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 8);
  return v;
}

// kMode 0: strided batch; 1: grouped launch, CTA i takes problem desc[i] (its
// own pointers and shape; the strided arguments are ignored); 2: as 1 with the
// range guard checked on every global access.
template <int kMode>
__global__ void __launch_bounds__(kThreads, 2) k_svd_left(const float* __restrict__ Kg_,
                                                           long long sK, int m_, int n_,
                                                           float* __restrict__ Ug_, long long sU,
                                                           float* __restrict__ Utg_, long long sUt,
                                                           double* __restrict__ lamg_,
                                                           long long slam, int r_, int nlam_,
                                                           int* __restrict__ status_, int rounds,
                                                           const SvdDesc* __restrict__ desc) {
  extern __shared__ __align__(16) float sm[];
  const SvdDesc* dq = kMode ? desc + blockIdx.x : nullptr;
  const GuardTab* gd = kMode == 2 ? dq->guard : nullptr;
  const float* Kg = dq ? dq->K : Kg_;
  float* Ug = dq ? dq->U : Ug_;
  float* Utg = dq ? dq->Ut : Utg_;
  double* lamg = dq ? dq->lam : lamg_;
  int* status = dq ? dq->status : status_;
  const int m = dq ? dq->m : m_, n = dq ? dq->n : n_, r = dq ? dq->r : r_;
  const int nlam = dq ? dq->nlam : nlam_;
  const int b = dq ? 0 : int(blockIdx.x);
  const int p = m < n ? m : n;
  const int N = (m < n) ? 2 * p + 1 : 2 * p;
  const int mr = (m + 3) & ~3;
  float* Refl = sm;                                   // packed left reflectors
  float* Zs = Refl + ((refl_total(m, p) + 3) & ~3);   // r x kRld: u parts of T_GK vectors
  float* Xc = Zs + r * kRld;                          // 2 x 128: published column
  float* Xr = Xc + 256;                               // 2 x 128: published row
  float* Wp = Xr + 256;                               // 8 x 128: per-warp u^T K partials
  float* dd = Wp + 1024;                              // diagonal of B
  float* ee = dd + kNmax;                             // superdiagonal of B
  float* tau = ee + kNmax;                            // left reflector scalars
  float* lam = tau + kNmax;                           // sigma, descending
  float* e2 = lam + kNmax;                            // 256: squared T_GK off-diagonals
  float* gk = e2 + 2 * kNmax;                         // 256: the off-diagonals
  int* gcnt = reinterpret_cast<int*>(gk + 2 * kNmax);  // 256
  float* pub = reinterpret_cast<float*>(gcnt + 2 * kNmax);  // 2 x kRld
  float* shift = pub + 2 * kRld;                      // 64
  float* scal = shift + 64;                           // 16
  int* roff = reinterpret_cast<int*>(scal + 16);      // 132: reflector offsets
  float* Zb = reinterpret_cast<float*>(roff + 132);   // 128: per-warp row sums
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ta = 2 * warp + (lane >> 4), tb = lane & 15;
  const int r0 = 8 * ta, c0 = 8 * tb;
  const float* K = Kg + (long long)b * sK;

  // ---- load the tile, screen for NaN/Inf
  float kt[8][8];
  bool bad = false;
#pragma unroll
  for (int ii = 0; ii < 8; ++ii)
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
      const int row = r0 + ii, col = c0 + jj;
      const float x = (row < m && col < n && guard_ok(gd, K + (long long)row * n + col, 4, 0x501))
                          ? K[(long long)row * n + col]
                          : 0.f;
      if (!isfinite(x)) bad = true;
      kt[ii][jj] = x;
    }
  if (tid == 0) {
    int t = 0;
    for (int k = 0; k < p; ++k) {
      roff[k] = t;
      t += refl_len(k, m);
    }
  }
  if (__syncthreads_or(bad)) {
    for (int idx = tid; idx < m * r; idx += kThreads)
      if (guard_ok(gd, Ug + (long long)b * sU + idx, 4, 0x502)) Ug[(long long)b * sU + idx] = 0.f;
    if (Utg)
      for (int idx = tid; idx < m * r; idx += kThreads)
        if (guard_ok(gd, Utg + (long long)b * sUt + idx, 4, 0x503))
          Utg[(long long)b * sUt + idx] = 0.f;
    if (lamg)
      for (int t = tid; t < nlam; t += kThreads)
        if (guard_ok(gd, lamg + (long long)b * slam + t, 8, 0x504))
          lamg[(long long)b * slam + t] = 0.0;
    if (tid == 0 && guard_ok(gd, status + b, 4, 0x505)) status[b] = TN_ERR_NONFINITE;
    return;
  }
  // publish column 0 and row 0
  if (tb == 0)
#pragma unroll
    for (int ii = 0; ii < 8; ++ii) Xc[r0 + ii] = kt[ii][0];
  if (ta == 0)
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) Xr[c0 + jj] = kt[0][jj];
  __syncthreads();

  // ---- a. Golub-Kahan bidiagonalisation.  A warp whose rows all lie above
  // row k has nothing left to do but meet the barriers; warp 7 (rows 112 ..
  // 127) is never idle and records d_k, e_k and tau_k.
  for (int k = 0; k < p; ++k) {
    const float* xc = Xc + (k & 1) * 128;
    const float* xr = Xr + (k & 1) * 128;
    const bool wact = 16 * warp + 15 >= k;  // warp-uniform
    float u[8], tk = 0.f;
    if (wact) {
      // left reflector from column k (every warp, same values)
      float sc;
      {
        const float4 x4 = *reinterpret_cast<const float4*>(xc + 4 * lane);
        const int i0 = 4 * lane;
        float t = (i0 > k && i0 < m) ? x4.x * x4.x : 0.f;
        t = (i0 + 1 > k && i0 + 1 < m) ? fmaf(x4.y, x4.y, t) : t;
        t = (i0 + 2 > k && i0 + 2 < m) ? fmaf(x4.z, x4.z, t) : t;
        t = (i0 + 3 > k && i0 + 3 < m) ? fmaf(x4.w, x4.w, t) : t;
        const float s = warp_sum(t);
        float beta;
        house(xc[k], s, beta, tk, sc);
        if (warp == 7 && lane == 0) {
          dd[k] = beta;
          tau[k] = tk;
        }
      }
      {
        const float4 xa = *reinterpret_cast<const float4*>(xc + r0);
        const float4 xb = *reinterpret_cast<const float4*>(xc + r0 + 4);
        const float xv[8] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
#pragma unroll
        for (int ii = 0; ii < 8; ++ii) {
          const int row = r0 + ii;
          u[ii] = (row == k) ? 1.f : ((row > k && row < m) ? xv[ii] * sc : 0.f);
        }
      }
      if (tb == 0) {  // keep reflector k for the back-transformation
        const int P0 = k & ~3;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int row = r0 + 4 * h;
          if (row >= P0 && row < mr)
            *reinterpret_cast<float4*>(Refl + roff[k] + rpad(row) - rpad(P0)) =
                make_float4(u[4 * h], u[4 * h + 1], u[4 * h + 2], u[4 * h + 3]);
        }
      }
      // column sums u^T K over this warp's two tile rows (packed FMAs)
      float2 cp[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) cp[q] = make_float2(0.f, 0.f);
#pragma unroll
      for (int ii = 0; ii < 8; ++ii) {
        const float2 uu = make_float2(u[ii], u[ii]);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          cp[q] = __ffma2_rn(uu, make_float2(kt[ii][2 * q], kt[ii][2 * q + 1]), cp[q]);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        cp[q].x += __shfl_xor_sync(0xffffffffu, cp[q].x, 16);
        cp[q].y += __shfl_xor_sync(0xffffffffu, cp[q].y, 16);
      }
      if (lane < 16) {  // [warp][half][tile column][4]: conflict-free float4 rows
        *reinterpret_cast<float4*>(Wp + warp * 128 + 4 * tb) =
            make_float4(cp[0].x, cp[0].y, cp[1].x, cp[1].y);
        *reinterpret_cast<float4*>(Wp + warp * 128 + 64 + 4 * tb) =
            make_float4(cp[2].x, cp[2].y, cp[3].x, cp[3].y);
      }
    }
    __syncthreads();
    if (wact) {
      // w = tau K^T u and the updated row k, y = K[k][.] - w, for this
      // thread's columns (the same sums in every thread of a tile column)
      float w[8], y[8];
      {
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) w[jj] = 0.f;
        const int wmin = k >> 4;
#pragma unroll
        for (int ww = 0; ww < 8; ++ww) {
          if (ww < wmin) continue;
          const float4 pa = *reinterpret_cast<const float4*>(Wp + ww * 128 + 4 * tb);
          const float4 pb = *reinterpret_cast<const float4*>(Wp + ww * 128 + 64 + 4 * tb);
          w[0] += pa.x; w[1] += pa.y; w[2] += pa.z; w[3] += pa.w;
          w[4] += pb.x; w[5] += pb.y; w[6] += pb.z; w[7] += pb.w;
        }
        const float4 ra = *reinterpret_cast<const float4*>(xr + c0);
        const float4 rb = *reinterpret_cast<const float4*>(xr + c0 + 4);
        const float rv[8] = {ra.x, ra.y, ra.z, ra.w, rb.x, rb.y, rb.z, rb.w};
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
          const int col = c0 + jj;
          const bool on = col > k && col < n;
          w[jj] = on ? tk * w[jj] : 0.f;
          y[jj] = on ? rv[jj] - w[jj] : 0.f;
        }
      }
      // right reflector from y over columns k+1 .. n-1 (every half warp,
      // same values)
      float tq = 0.f, sc2 = 0.f;
      {
        float t = 0.f;
#pragma unroll
        for (int jj = 0; jj < 8; ++jj)
          if (c0 + jj > k + 1) t = fmaf(y[jj], y[jj], t);
        const float s2 = half_sum(t);
        float yk1 = 0.f;
        switch ((k + 1) & 7) {  // uniform: a static register index per case
          case 0: yk1 = y[0]; break;
          case 1: yk1 = y[1]; break;
          case 2: yk1 = y[2]; break;
          case 3: yk1 = y[3]; break;
          case 4: yk1 = y[4]; break;
          case 5: yk1 = y[5]; break;
          case 6: yk1 = y[6]; break;
          default: yk1 = y[7]; break;
        }
        const float alpha2 = __shfl_sync(0xffffffffu, yk1, (((k + 1) >> 3) & 15) + (lane & 16));
        float beta2 = 0.f;
        if (k + 1 < n) house(alpha2, s2, beta2, tq, sc2);
        if (warp == 7 && lane == 0) ee[k] = beta2;
      }
      float v[8];
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) {
        const int col = c0 + jj;
        v[jj] = (col == k + 1 && k + 1 < n) ? 1.f : ((col > k + 1 && col < n) ? y[jj] * sc2 : 0.f);
      }
      float wv = 0.f;
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) wv = fmaf(w[jj], v[jj], wv);
      wv = half_sum(wv);
      // row sums K v over a tile row: packed FMAs, then a reduce-scatter over
      // the sixteen lanes (lane pair (b, b ^ 1) ends with row 4 b3 + 2 b2 + b1
      // of the tile) and a gather through shared memory
      float z[8];
      {
        float t[8];
#pragma unroll
        for (int ii = 0; ii < 8; ++ii) {
          float2 acc = make_float2(0.f, 0.f);
#pragma unroll
          for (int q = 0; q < 4; ++q)
            acc = __ffma2_rn(make_float2(kt[ii][2 * q], kt[ii][2 * q + 1]),
                             make_float2(v[2 * q], v[2 * q + 1]), acc);
          t[ii] = acc.x + acc.y;
        }
        const bool h3 = tb & 8, h2 = tb & 4, h1 = tb & 2;
        float a4[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float send = h3 ? t[i] : t[i + 4];
          const float keep = h3 ? t[i + 4] : t[i];
          a4[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
        }
        float a2[2];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          const float send = h2 ? a4[i] : a4[i + 2];
          const float keep = h2 ? a4[i + 2] : a4[i];
          a2[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
        }
        float a1;
        {
          const float send = h1 ? a2[0] : a2[1];
          const float keep = h1 ? a2[1] : a2[0];
          a1 = keep + __shfl_xor_sync(0xffffffffu, send, 2);
        }
        a1 += __shfl_xor_sync(0xffffffffu, a1, 1);
        float* zb = Zb + warp * 16 + (lane >> 4) * 8;
        if ((tb & 1) == 0) zb[(h3 ? 4 : 0) + (h2 ? 2 : 0) + (h1 ? 1 : 0)] = a1;
        __syncwarp();
        const float4 za = *reinterpret_cast<const float4*>(zb);
        const float4 zc = *reinterpret_cast<const float4*>(zb + 4);
        const float zr[8] = {za.x, za.y, za.z, za.w, zc.x, zc.y, zc.z, zc.w};
#pragma unroll
        for (int ii = 0; ii < 8; ++ii) {
          const int row = r0 + ii;
          z[ii] = (row > k) ? tq * fmaf(-u[ii], wv, zr[ii]) : 0.f;
        }
      }
      // K -= u w^T + z v^T (packed FMAs)
      if (r0 + 7 > k && c0 + 7 > k) {
#pragma unroll
        for (int ii = 0; ii < 8; ++ii) {
          const float2 nu = make_float2(-u[ii], -u[ii]), nz = make_float2(-z[ii], -z[ii]);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            float2 x = __ffma2_rn(nu, make_float2(w[2 * q], w[2 * q + 1]),
                                  make_float2(kt[ii][2 * q], kt[ii][2 * q + 1]));
            x = __ffma2_rn(nz, make_float2(v[2 * q], v[2 * q + 1]), x);
            kt[ii][2 * q] = x.x;
            kt[ii][2 * q + 1] = x.y;
          }
        }
      }
    }
    // publish column k+1 and row k+1 for the next step (rows above k + 1,
    // held by idle warps, are masked by every reader)
    if (k + 1 < p && wact) {
      const int cn = k + 1;
      float* xcn = Xc + (cn & 1) * 128;
      float* xrn = Xr + (cn & 1) * 128;
      if (tb == (cn >> 3)) {
        switch (cn & 7) {
#define TN_PUB_COL(E) \
  case E: {           \
    _Pragma("unroll") for (int ii = 0; ii < 8; ++ii) xcn[r0 + ii] = kt[ii][E]; \
  } break;
          TN_PUB_COL(0) TN_PUB_COL(1) TN_PUB_COL(2) TN_PUB_COL(3)
          TN_PUB_COL(4) TN_PUB_COL(5) TN_PUB_COL(6) TN_PUB_COL(7)
#undef TN_PUB_COL
        }
      }
      if (ta == (cn >> 3)) {
        switch (cn & 7) {
#define TN_PUB_ROW(E)                                                            \
  case E: {                                                                      \
    *reinterpret_cast<float4*>(xrn + c0) =                                       \
        make_float4(kt[E][0], kt[E][1], kt[E][2], kt[E][3]);                     \
    *reinterpret_cast<float4*>(xrn + c0 + 4) =                                   \
        make_float4(kt[E][4], kt[E][5], kt[E][6], kt[E][7]);                     \
  } break;
          TN_PUB_ROW(0) TN_PUB_ROW(1) TN_PUB_ROW(2) TN_PUB_ROW(3)
          TN_PUB_ROW(4) TN_PUB_ROW(5) TN_PUB_ROW(6) TN_PUB_ROW(7)
#undef TN_PUB_ROW
        }
      }
    }
    __syncthreads();
  }

  // ---- Golub-Kahan tridiagonal: off-diagonals g = d_0, e_0, d_1, e_1, ...
  if (tid < N - 1) {
    const int i = tid >> 1;
    const float g = (tid & 1) ? ee[i] : dd[i];
    gk[tid] = g;
    e2[tid] = g * g;
  }
  __syncthreads();
  if (tid == 0) {
    float gu = 0.f, emax = 0.f;
    for (int j = 0; j < N; ++j) {
      const float gl_ = (j > 0) ? fabsf(gk[j - 1]) : 0.f;
      const float gr_ = (j + 1 < N) ? fabsf(gk[j]) : 0.f;
      gu = fmaxf(gu, gl_ + gr_);
      if (j + 1 < N) emax = fmaxf(emax, e2[j]);
    }
    const float eps = FLT_EPSILON * 0.5f;
    const float pivmin = FLT_MIN * fmaxf(1.f, emax);
    const float pad = 2.1f * gu * eps * float(N) + 4.2f * pivmin;
    scal[2] = -gu - pad;
    scal[3] = gu + pad;
    scal[4] = gu;
    scal[5] = pivmin;
  }
  __syncthreads();
  const float gl = scal[2], gu = scal[3], tnorm = scal[4], pivmin = scal[5];
  const float eps = FLT_EPSILON * 0.5f;

  // ---- b. multisection for the nl largest eigenvalues of T_GK
  const int nl = min(max(nlam, r), p);
  {
    const int q = tid & 3;
    const float hg = (gu - gl) / float(kThreads + 1);
    gcnt[tid] = sturm_gk(e2, N, fmaf(hg, float(tid + 1), gl), pivmin);
    __syncthreads();
    for (int base = 0; base < nl; base += kThreads / 4) {
      const int t = base + (tid >> 2);
      const bool valid = t < nl;
      const int j = N - 1 - t;  // ascending index of the t-th largest
      int m0 = 0, m1 = kThreads;
      for (int it = 0; it < 9; ++it) {
        if (m0 >= m1) break;
        const int mid = (m0 + m1) >> 1;
        if (gcnt[mid] <= j) m0 = mid + 1;
        else m1 = mid;
      }
      float lo = (m0 > 0) ? fmaf(hg, float(m0), gl) : gl;
      float hi = (m0 < kThreads) ? fmaf(hg, float(m0 + 1), gl) : gu;
      for (int it = 0; it < rounds; ++it) {
        const float h = (hi - lo) / 5.f;
        const float x = fmaf(h, float(q + 1), lo);
        const int cnt = valid ? sturm_gk(e2, N, x, pivmin) : 0;
        int mm = (valid && cnt <= j) ? 1 : 0;
        mm += __shfl_xor_sync(0xffffffffu, mm, 1);
        mm += __shfl_xor_sync(0xffffffffu, mm, 2);
        const float nlo = (mm > 0) ? fmaf(h, float(mm), lo) : lo;
        hi = (mm < 4) ? fmaf(h, float(mm + 1), lo) : hi;
        lo = nlo;
      }
      if (valid && q == 0) {
        lam[t] = fmaxf(0.5f * (lo + hi), 0.f);
        if (hi - lo > 128.f * eps * tnorm && guard_ok(gd, status + b, 4, 0x506))
          atomicCAS(status + b, 0, int(TN_ERR_EIG_NOCONV));
      }
    }
  }
  __syncthreads();
  if (tid == 0) {
    const float pertol = 10.f * eps * fmaxf(tnorm, FLT_MIN);
    for (int t = 0; t < r; ++t) {
      float s = lam[t];
      if (t > 0 && shift[t - 1] - s < pertol) s = shift[t - 1] - pertol;
      shift[t] = s;
    }
  }
  __syncthreads();

  // ---- c. inverse iteration on T_GK - sigma I, one thread per vector, two
  // solves from a fixed pseudo-random start; solution and triangular factor
  // (rows divided by their pivots) in local memory; the odd entries (the
  // left singular vector of B), max-abs normalised, go to the thread's padded
  // row of Zs
  if (tid < r) {
    float y[2 * kNmax + 1], u2[2 * kNmax + 1], u3[2 * kNmax + 1];
    auto start = [&](int i) {
      unsigned int hsh = 2654435761u * (unsigned)(i + 1) ^ (40503u * (unsigned)(tid + 7));
      hsh ^= hsh >> 13; hsh *= 0x5bd1e995u; hsh ^= hsh >> 15;
      return 1.f + 0.5f * (float(hsh & 0xffff) / 65536.f - 0.5f);
    };
    const float lmb = shift[tid];
    const float tp = fmaxf(eps * tnorm, FLT_MIN);
    float inv = 1.f;
    for (int it = 0; it < 2; ++it) {
      float a = -lmb;
      float bb = (N > 1) ? gk[0] : 0.f;
      float yk = (it == 0) ? start(0) : y[0] * inv;
      for (int i0 = 0; i0 + 1 < N; i0 += 8) {
        float yg[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int i = i0 + q;
          yg[q] = (i + 1 < N) ? ((it == 0) ? start(i + 1) : y[i + 1] * inv) : 0.f;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int i = i0 + q;
          if (i + 1 >= N) break;
          const float c = gk[i];
          const float ns = (i + 2 < N) ? gk[i + 1] : 0.f;
          const bool piv = fabsf(a) >= fabsf(c);
          const float den = piv ? ((a == 0.f) ? tp : a) : c;
          const float rd = __fdividef(1.f, den);
          const float mlt = (piv ? c : a) * rd;
          const float yo = piv ? yk : yg[q], ye = piv ? yg[q] : yk;
          u2[i] = (piv ? bb : -lmb) * rd;
          u3[i] = piv ? 0.f : ns * rd;
          y[i] = yo * rd;
          yk = fmaf(-mlt, yo, ye);
          a = piv ? fmaf(-mlt, bb, -lmb) : fmaf(-mlt, -lmb, bb);
          bb = piv ? ns : -mlt * ns;
        }
      }
      if (a == 0.f) a = tp;
      float x2 = __fdividef(yk, a);
      y[N - 1] = x2;
      float x1 = x2;
      float mx = fabsf(x2);
      if (N >= 2) {
        x1 = fmaf(-u2[N - 2], x2, y[N - 2]);
        y[N - 2] = x1;
        mx = fmaxf(mx, fabsf(x1));
      }
      for (int i0 = N - 3; i0 >= 0; i0 -= 8) {
        float yg[8], ag[8], bg[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int i = i0 - q;
          yg[q] = (i >= 0) ? y[i] : 0.f;
          ag[q] = (i >= 0) ? u2[i] : 0.f;
          bg[q] = (i >= 0) ? u3[i] : 0.f;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int i = i0 - q;
          if (i < 0) break;
          const float xi = yg[q] - ag[q] * x1 - bg[q] * x2;
          y[i] = xi;
          mx = fmaxf(mx, fabsf(xi));
          x2 = x1;
          x1 = xi;
        }
      }
      inv = (mx > 0.f && isfinite(mx)) ? 1.f / mx : 1.f;
    }
    float* zo = Zs + tid * kRld;
    for (int i = 0; i < p; ++i) zo[rpad(i)] = y[2 * i + 1] * inv;
    for (int i = p; i < kNmax; ++i) zo[rpad(i)] = 0.f;
  }
  __syncthreads();

  // ---- d. vectors: thread quad (column col, quarter qr), rows 32 qr + kk
  const int col = tid >> 2, qr = tid & 3;
  const bool live = col < r;
  float z[kQ];
  auto load32 = [&](const float* src, float* dst) {
#pragma unroll
    for (int mm = 0; mm < kQ / 4; ++mm) {
      const float4 t = *reinterpret_cast<const float4*>(src + qr * 36 + 4 * mm);
      dst[4 * mm] = t.x; dst[4 * mm + 1] = t.y; dst[4 * mm + 2] = t.z; dst[4 * mm + 3] = t.w;
    }
  };
  if (live) load32(Zs + col * kRld, z);
  else
#pragma unroll
    for (int kk = 0; kk < kQ; ++kk) z[kk] = 0.f;
  auto dot32 = [](const float* x, const float* y2) {
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
    for (int kk = 0; kk < kQ; kk += 4) {
      a0 = fmaf(x[kk], y2[kk], a0);
      a1 = fmaf(x[kk + 1], y2[kk + 1], a1);
      a2 = fmaf(x[kk + 2], y2[kk + 2], a2);
      a3 = fmaf(x[kk + 3], y2[kk + 3], a3);
    }
    return (a0 + a1) + (a2 + a3);
  };
  auto normalise_publish = [&](float* dst) {
    const float s = quad_sum(dot32(z, z));
    const float iv = (s > 0.f) ? 1.f / sqrtf(s) : 0.f;
#pragma unroll
    for (int kk = 0; kk < kQ; ++kk) z[kk] *= iv;
#pragma unroll
    for (int mm = 0; mm < kQ / 4; ++mm)
      *reinterpret_cast<float4*>(dst + qr * 36 + 4 * mm) =
          make_float4(z[4 * mm], z[4 * mm + 1], z[4 * mm + 2], z[4 * mm + 3]);
  };
  // Modified Gram-Schmidt, run twice ("twice is enough", Kahan-Parlett):
  // singular values at the FP32 resolution of K come out of inverse
  // iteration as nearly parallel vectors, and one pass leaves them orthogonal
  // only to eps / |residual|.
  for (int pass = 0; pass < 2; ++pass) {
    __syncthreads();  // the previous pass's reads of both buffers are done
    if (col == 0) normalise_publish(pub);
    for (int j = 0; j < r; ++j) {
      __syncthreads();  // vector j published; reads of the other buffer done
      if (live && col > j) {
        float pj[kQ];
        load32(pub + (j & 1) * kRld, pj);
        const float d = quad_sum(dot32(pj, z));
#pragma unroll
        for (int kk = 0; kk < kQ; ++kk) z[kk] = fmaf(-d, pj[kk], z[kk]);
        if (col == j + 1) normalise_publish(pub + ((j + 1) & 1) * kRld);
      }
    }
  }
  if (live) {
    // U = H_0 ... H_{p-1} [u; 0]
    for (int k = p - 1; k >= 0; --k) {
      const float tk = tau[k];
      if (tk == 0.f) continue;
      const int P0 = k & ~3;
      const float* rk = Refl + roff[k] - rpad(P0);
      float vk[kQ];
#pragma unroll
      for (int mm = 0; mm < kQ / 4; ++mm) {
        const int row = 32 * qr + 4 * mm;
        float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
        if (row >= P0 && row < mr) t = *reinterpret_cast<const float4*>(rk + qr * 36 + 4 * mm);
        vk[4 * mm] = t.x; vk[4 * mm + 1] = t.y; vk[4 * mm + 2] = t.z; vk[4 * mm + 3] = t.w;
      }
      const float d = quad_sum(dot32(vk, z)) * tk;
#pragma unroll
      for (int kk = 0; kk < kQ; ++kk) z[kk] = fmaf(-d, vk[kk], z[kk]);
    }
    const unsigned qm = 0xFu << (threadIdx.x & 28);
    {
      // unit norm to FP32 rounding: the reflectors, applied in FP32, leave
      // |u| = 1 + O(p eps) with a bias of one sign, which would compound over
      // the vertices of a pass and over passes (each pass's network is the
      // previous tree); the norm is summed in FP64
      double s2 = 0.0;
#pragma unroll
      for (int kk = 0; kk < kQ; ++kk) s2 = fma(double(z[kk]), double(z[kk]), s2);
      for (int o = 1; o <= 2; o <<= 1) s2 += __shfl_xor_sync(qm, s2, o);
      const float iv = (s2 > 0.0) ? float(1.0 / sqrt(s2)) : 0.f;
#pragma unroll
      for (int kk = 0; kk < kQ; ++kk) z[kk] *= iv;
    }
    float best = -1.f;
    int bi = kNmax;
#pragma unroll
    for (int kk = 0; kk < kQ; ++kk) {
      const int row = 32 * qr + kk;
      const float av = fabsf(z[kk]);
      if (row < m && (av > best || (av == best && row < bi))) { best = av; bi = row; }
    }
    for (int o = 1; o <= 2; o <<= 1) {
      const float ob = __shfl_xor_sync(qm, best, o);
      const int oi = __shfl_xor_sync(qm, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    float sv = 0.f;
#pragma unroll
    for (int kk = 0; kk < kQ; ++kk)
      if (32 * qr + kk == bi) sv = z[kk];
    sv = quad_sum(sv);
    const float sg = (sv < 0.f) ? -1.f : 1.f;
    float* U = Ug + (long long)b * sU;
    float* Ut = Utg ? Utg + (long long)b * sUt + (long long)col * m : nullptr;
#pragma unroll
    for (int kk = 0; kk < kQ; ++kk) {
      const int row = 32 * qr + kk;
      if (row < m) {
        if (guard_ok(gd, U + (long long)row * r + col, 4, 0x507))
          U[(long long)row * r + col] = sg * z[kk];
        if (Ut && guard_ok(gd, Ut + row, 4, 0x508)) Ut[row] = sg * z[kk];
      }
    }
  }
  if (lamg) {
    double* lo = lamg + (long long)b * slam;
    for (int t = tid; t < nlam; t += kThreads) {
      const double sv = (t < nl) ? double(lam[t]) : 0.0;
      if (guard_ok(gd, lo + t, 8, 0x509)) lo[t] = sv * sv;
    }
  }
}

}  // namespace

cudaError_t launch_chol_env(float* R, long long sR, const int64_t* r_off, const int32_t* D,
                            int maxD, const unsigned int* amax, long long s_amax, int k0, int nk,
                            int batch, cudaStream_t st) {
  if (maxD < 1 || maxD > kNmax || nk < 1) return cudaErrorInvalidValue;
  k_chol_env<0><<<batch * nk, kThreads, 0, st>>>(R, sR, r_off, D, amax, s_amax, k0, nk, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_chol_grouped(const CholDesc* desc, int n_prob, bool guarded, cudaStream_t st) {
  if (n_prob <= 0) return cudaSuccess;
  if (guarded)
    k_chol_env<2><<<n_prob, kThreads, 0, st>>>(nullptr, 0, nullptr, nullptr, nullptr, 0, 0, 1, desc);
  else
    k_chol_env<1><<<n_prob, kThreads, 0, st>>>(nullptr, 0, nullptr, nullptr, nullptr, 0, 0, 1, desc);
  return cudaGetLastError();
}

size_t svd_left_smem_bytes(int m, int n, int r) {
  const int p = m < n ? m : n;
  return sizeof(float) *
         (size_t((refl_total(m, p) + 3) & ~3) + size_t(r) * kRld + size_t(kSmallFloats));
}

bool svd_left_supported(int m, int n, int r) {
  return m >= 1 && n >= 1 && m <= kNmax && n <= kNmax && r >= 1 && r <= kRmax &&
         r <= (m < n ? m : n);
}

cudaError_t launch_svd_left(const float* K, long long sK, int m, int n, float* U, long long sU,
                            float* Ut, long long sUt, double* lam, long long slam, int r,
                            int nlam, int* status, int batch, cudaStream_t st, int rounds) {
  if (!svd_left_supported(m, n, r) || nlam < 0 || nlam > m || rounds < 1 || rounds > 16)
    return cudaErrorInvalidValue;
  const size_t smem = svd_left_smem_bytes(m, n, r);
  k_svd_left<0><<<batch, kThreads, smem, st>>>(K, sK, m, n, U, sU, Ut, sUt, lam, slam, r, nlam,
                                            status, rounds, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_svd_left_grouped(const SvdDesc* desc, int n_prob, int max_m, int max_n,
                                    int max_r, bool guarded, cudaStream_t st, int rounds) {
  if (n_prob <= 0) return cudaSuccess;
  if (!svd_left_supported(max_m, max_n, max_r) || rounds < 1 || rounds > 16)
    return cudaErrorInvalidValue;
  const size_t smem = svd_left_smem_bytes(max_m, max_n, max_r);
  auto kern = guarded ? k_svd_left<2> : k_svd_left<1>;
  kern<<<n_prob, kThreads, smem, st>>>(nullptr, 0, 0, 0, nullptr, 0, nullptr, 0, nullptr, 0,
                                             0, 0, nullptr, rounds, desc);
  return cudaGetLastError();
}

cudaError_t svd_configure() {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  const size_t need_svd = svd_left_smem_bytes(kNmax, kNmax, kRmax);
  if (need_svd > size_t(optin)) return cudaErrorInvalidValue;
  for (auto kern : {k_svd_left<0>, k_svd_left<1>, k_svd_left<2>}) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(need_svd));
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace tn
