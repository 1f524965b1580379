// Factored density matrices of the mixed-precision path.
//
// Algorithm density_matrix_alg (Sec. 5) keeps the leading eigenvectors of
// L_v = M_v R_v M_v^T, with R_v the memoised root-side density matrix of
// Eq. dm_cache.  Forming L_v in FP32 squares the conditioning of M_v: its
// rounding (~6e-8 of the largest eigenvalue) drowns every eigen-direction
// below that level, and a truncation that falls there picks a subspace that
// does not belong to the stored state.  This file never forms L_v:
//   1. k_chol_env: R_v = C_v C_v^T (FP32 Cholesky, one CTA per R_v, every
//      R_v of a pass in one launch; a non-positive pivot gives a zero column,
//      so rank-deficient environments need no shift);
//   2. K_v = M_v C_v on the tensor cores (compensated TF32, elsewhere);
//   3. k_svd_left: the leading left singular vectors of K_v, which are the
//      leading eigenvectors of L_v = K_v K_v^T, and sigma^2 as its
//      eigenvalues.  Backward error eps ||K_v|| on K_v is eps^2 ||L_v|| on
//      the density matrix.
// The SVD follows the bisection-and-inverse-iteration route of Marques,
// Demmel and Vasconcelos (LAPACK xBDSVDX):
//   a. Golub-Kahan bidiagonalisation K = H B G^T by Householder reflectors
//      (Golub & Van Loan, Matrix Computations, Sec. 5.4.8), K in shared
//      memory, left reflectors kept, right reflectors dropped;
//   b. the r largest eigenvalues of the Golub-Kahan tridiagonal T_GK (zero
//      diagonal, off-diagonals d_0, e_0, d_1, e_1, ...; eigenvalues
//      +-sigma_i) by Sturm-sequence multisection;
//   c. eigenvectors of T_GK by inverse iteration with partial pivoting; the
//      entries at odd positions are the left singular vector of B;
//   d. modified Gram-Schmidt, back-transformation U = H_0 ... H_{p-1} [u; 0],
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
// One CTA per (instance, tree vertex k): R = R_k / max|R_k| (symmetrised),
// right-looking unblocked Cholesky R = C C^T in FP32.  Step j reads column j
// and the pivot, both final since step j - 1, and updates the trailing lower
// triangle; column j is scaled only at the store.  A pivot that is not
// positive (round-off of a semi-definite R) leaves column j zero and the
// trailing block untouched.  Output in place of R_k: B[j][l] = C[l][j]
// (row-major, upper triangular), the K-major second operand of K = M C.
__global__ void __launch_bounds__(kThreads) k_chol_env(float* __restrict__ R, long long sR,
                                                        const int64_t* __restrict__ r_off,
                                                        const int32_t* __restrict__ D,
                                                        const unsigned int* __restrict__ amax,
                                                        long long s_amax, int k0, int nk) {
  extern __shared__ __align__(16) float ch[];
  const int b = blockIdx.x / nk;
  const int k = k0 + blockIdx.x % nk;
  const int n = D[k];
  const int ld = n | 1;  // odd pitch: column reads hit distinct banks
  float* A = ch;
  float* rs = ch + n * ld;  // 1 / sqrt(pivot), or 0
  float* Rg = R + (long long)b * sR + r_off[k];
  const float am = __uint_as_float(amax[(long long)b * s_amax + k]);
  const float sc = (am > 0.f && isfinite(am)) ? 1.f / am : 1.f;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < n * n; idx += kThreads) {
    const int i = idx / n, j = idx - i * n;
    A[i * ld + j] = Rg[idx] * sc;
  }
  __syncthreads();
  for (int idx = tid; idx < n * n; idx += kThreads) {
    const int i = idx / n, j = idx - i * n;
    if (j < i) {
      const float x = 0.5f * (A[i * ld + j] + A[j * ld + i]);
      A[i * ld + j] = x;  // lower triangle only from here on
    }
  }
  __syncthreads();
  // thread pair per row: row i = k + 1 + (tid >> 1) (+128 for the second
  // pass), the two lanes take alternate columns
  for (int j = 0; j < n; ++j) {
    const float p = A[j * ld + j];
    if (p > 0.f && isfinite(p)) {
      const float ip = 1.f / p;
      for (int i = j + 1 + (tid >> 1); i < n; i += kThreads / 2) {
        const float aij = A[i * ld + j] * ip;
        for (int c = j + 1 + (tid & 1); c <= i; c += 2) A[i * ld + c] -= aij * A[c * ld + j];
      }
    }
    __syncthreads();
  }
  for (int j = tid; j < n; j += kThreads) {
    const float p = A[j * ld + j];
    rs[j] = (p > 0.f && isfinite(p)) ? 1.f / sqrtf(p) : 0.f;
  }
  __syncthreads();
  for (int idx = tid; idx < n * n; idx += kThreads) {
    const int j = idx / n, l = idx - j * n;  // B[j][l] = C[l][j]
    float v = 0.f;
    if (l > j) v = A[l * ld + j] * rs[j];
    else if (l == j) v = (rs[j] > 0.f) ? A[j * ld + j] * rs[j] : 0.f;
    Rg[idx] = v;
  }
}

// ---------------------------------------------------------------- SVD
// Shared layout (floats): a region of max(m * ldk, r * zld) holding K during
// the bidiagonalisation and the Golub-Kahan vectors afterwards; the packed
// left reflectors (row k + 1 .. m - 1 of reflector k, back to back); then
// the 128/256-entry work vectors.
struct SvdLayout {
  int ldk, N, zld, region, refl;
};

__host__ __device__ inline SvdLayout svd_layout(int m, int n, int r) {
  SvdLayout L;
  L.ldk = n | 1;
  const int p = m < n ? m : n;
  L.N = (m < n) ? 2 * p + 1 : 2 * p;
  L.zld = L.N + 1;
  const int a = m * L.ldk, z = r * L.zld;
  L.region = ((a > z ? a : z) + 3) & ~3;
  L.refl = ((p * (m - 1) - (p * (p - 1)) / 2) + 3) & ~3;
  if (L.refl < 4) L.refl = 4;
  return L;
}

constexpr int kSmallFloats = 128 * 8 + 256 * 3 + 2 * 132 + 64 + 16;

__host__ __device__ inline int refl_off(int k, int m) { return k * (m - 1) - (k * (k - 1)) / 2; }

__device__ int sturm_gk(const float* e2, int N, float x, float pivmin) {
  // T_GK has a zero diagonal: q_0 = -x, q_j = -x - g_{j-1}^2 / q_{j-1}
  float q = -x;
  if (fabsf(q) < pivmin) q = -pivmin;
  int c = (q < 0.f);
  for (int j = 1; j < N; ++j) {
    q = -x - __fdividef(e2[j - 1], q);
    if (fabsf(q) < pivmin) q = -pivmin;
    c += (q < 0.f);
  }
  return c;
}

__global__ void __launch_bounds__(kThreads) k_svd_left(const float* __restrict__ Kg, long long sK,
                                                        int m, int n, float* __restrict__ Ug,
                                                        long long sU, float* __restrict__ Utg,
                                                        long long sUt, double* __restrict__ lamg,
                                                        long long slam, int r, int nlam,
                                                        int* __restrict__ status) {
  extern __shared__ __align__(16) float sm[];
  const SvdLayout Ly = svd_layout(m, n, r);
  const int p = m < n ? m : n;
  const int N = Ly.N, ldk = Ly.ldk, zld = Ly.zld;
  float* Kr = sm;                    // m x ldk, then r x zld (Golub-Kahan vectors)
  float* Refl = sm + Ly.region;      // packed left reflectors
  float* dd = Refl + Ly.refl;        // 128: diagonal of B
  float* ee = dd + kNmax;            // 128: superdiagonal of B
  float* tau = ee + kNmax;           // 128: left reflector scalars
  float* Uw = tau + kNmax;           // 128: current left reflector (zero outside k..m-1)
  float* W = Uw + kNmax;             // 128: tau K^T u, then row k of the updated K
  float* V = W + kNmax;              // 128: current right reflector (zero outside)
  float* Z = V + kNmax;              // 128: tau' (K - u w^T) v
  float* lam = Z + kNmax;            // 128: sigma, descending
  float* e2 = lam + kNmax;           // 256: squared Golub-Kahan off-diagonals
  float* gk = e2 + 2 * kNmax;        // 256: the off-diagonals themselves
  int* gcnt = reinterpret_cast<int*>(gk + 2 * kNmax);  // 256
  float* pub = reinterpret_cast<float*>(gcnt + 2 * kNmax);  // 2 x 132
  float* shift = pub + 2 * 132;      // 64
  float* scal = shift + 64;          // 16
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int b = blockIdx.x;
  const float* K = Kg + (long long)b * sK;

  // ---- load K, screen for NaN/Inf
  bool bad = false;
  for (int i = warp; i < m; i += kThreads / 32)
    for (int j = lane; j < n; j += 32) {
      const float x = K[(long long)i * n + j];
      if (!isfinite(x)) bad = true;
      Kr[i * ldk + j] = x;
    }
  if (__syncthreads_or(bad)) {
    for (int idx = tid; idx < m * r; idx += kThreads) Ug[(long long)b * sU + idx] = 0.f;
    if (Utg)
      for (int idx = tid; idx < m * r; idx += kThreads) Utg[(long long)b * sUt + idx] = 0.f;
    if (lamg)
      for (int t = tid; t < nlam; t += kThreads) lamg[(long long)b * slam + t] = 0.0;
    if (tid == 0) status[b] = TN_ERR_NONFINITE;
    return;
  }

  // ---- a. Golub-Kahan bidiagonalisation
  for (int k = 0; k < p; ++k) {
    // A: left reflector from column k, rows k .. m-1 (warp 0)
    if (warp == 0) {
      float s = 0.f;
      for (int i = k + 1 + lane; i < m; i += 32) {
        const float x = Kr[i * ldk + k];
        s = fmaf(x, x, s);
      }
      s = warp_sum(s);
      const float alpha = Kr[k * ldk + k];
      float tk, beta, sc;
      if (s == 0.f) {
        tk = 0.f; beta = alpha; sc = 0.f;
      } else {
        beta = -copysignf(sqrtf(alpha * alpha + s), alpha);
        tk = (beta - alpha) / beta;
        sc = 1.f / (alpha - beta);
      }
      const int ro = refl_off(k, m);
      for (int i = lane; i < kNmax; i += 32) {
        float u = 0.f;
        if (i == k) u = 1.f;
        else if (i > k && i < m && tk != 0.f) u = Kr[i * ldk + k] * sc;
        Uw[i] = u;
        if (i > k && i < m) Refl[ro + (i - k - 1)] = u;
      }
      if (lane == 0) {
        dd[k] = beta;
        tau[k] = tk;
      }
    }
    __syncthreads();
    // B: w_j = tau sum_i u_i K[i][j] (j > k), two threads per column with the
    // rows split in halves; W[j] = row k of the updated K, K[k][j] - w_j
    {
      const float tk = tau[k];
      const int j = tid >> 1, h = tid & 1;
      const int mid = (k + m + 1) >> 1;
      const int i0 = h ? mid : k, i1 = h ? m : mid;
      float s = 0.f;
      if (j > k && j < n && tk != 0.f)
        for (int i = i0; i < i1; ++i) s = fmaf(Uw[i], Kr[i * ldk + j], s);
      s += __shfl_xor_sync(0xffffffffu, s, 1);
      if (h == 0 && j < kNmax) {
        const float w = tk * s;
        Z[j] = (j > k && j < n) ? w : 0.f;  // w, kept for the update
        W[j] = (j > k && j < n) ? Kr[k * ldk + j] - w : 0.f;
      }
    }
    __syncthreads();
    // C: right reflector from row k, columns k+1 .. n-1 (warp 0); also w . v
    if (warp == 0) {
      float tq = 0.f, beta = 0.f, sc = 0.f;
      if (k + 1 < n) {
        float s = 0.f;
        for (int j = k + 2 + lane; j < n; j += 32) s = fmaf(W[j], W[j], s);
        s = warp_sum(s);
        const float alpha = W[k + 1];
        if (s == 0.f) {
          tq = 0.f; beta = alpha;
        } else {
          beta = -copysignf(sqrtf(alpha * alpha + s), alpha);
          tq = (beta - alpha) / beta;
          sc = 1.f / (alpha - beta);
        }
      }
      float wv = 0.f;
      for (int j = lane; j < kNmax; j += 32) {
        float v = 0.f;
        if (j == k + 1 && k + 1 < n) v = 1.f;
        else if (j > k + 1 && j < n && tq != 0.f) v = W[j] * sc;
        V[j] = v;
        wv = fmaf(Z[j], v, wv);
      }
      wv = warp_sum(wv);
      if (lane == 0) {
        ee[k] = beta;
        scal[0] = tq;
        scal[1] = wv;
      }
    }
    __syncthreads();
    // D: z_i = tau' (sum_j K[i][j] v_j - u_i (w . v)) for rows i > k, from
    // the matrix before this step's update; two threads per row
    const float tq = scal[0];
    float zi = 0.f;
    const int iz = k + 1 + (tid >> 1);
    if (tq != 0.f) {
      const int h = tid & 1;
      const int midc = (k + 1 + n + 1) >> 1;
      const int j0 = h ? midc : k + 1, j1 = h ? n : midc;
      float s = 0.f;
      if (iz < m)
        for (int j = j0; j < j1; ++j) s = fmaf(Kr[iz * ldk + j], V[j], s);
      s += __shfl_xor_sync(0xffffffffu, s, 1);
      zi = tq * (s - Uw[iz < kNmax ? iz : 0] * scal[1]);
    }
    __syncthreads();  // every read of K for z done; W, Z (w) stable
    // E: K[i][j] -= u_i w_j + z_i v_j for i, j > k; z_i travels through
    // shared memory (the w copy in Z is read first into registers)
    float wj[4], vj[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = lane + 32 * c;
      wj[c] = Z[j];
      vj[c] = V[j];
    }
    __syncthreads();
    if ((tid & 1) == 0 && iz < m) Z[iz] = zi;
    __syncthreads();
    for (int i = k + 1 + warp; i < m; i += kThreads / 32) {
      const float ui = Uw[i], zr = (tq != 0.f) ? Z[i] : 0.f;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int j = lane + 32 * c;
        if (j > k && j < n) {
          float x = Kr[i * ldk + j];
          x = fmaf(-ui, wj[c], x);
          x = fmaf(-zr, vj[c], x);
          Kr[i * ldk + j] = x;
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
      const float gl_ = (j > 0) ? sqrtf(e2[j - 1]) : 0.f;
      const float gr_ = (j + 1 < N) ? sqrtf(e2[j]) : 0.f;
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
      for (int it = 0; it < 10; ++it) {
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
      if (valid && q == 0) lam[t] = fmaxf(0.5f * (lo + hi), 0.f);
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
  // solves from a fixed pseudo-random start; the solution lives in this
  // thread's column of the region (K is no longer needed), the triangular
  // factor (rows divided by their pivots) in local memory
  float* Zs = Kr;
  if (tid < r) {
    float u2[2 * kNmax + 1], u3[2 * kNmax + 1];
    float* y = Zs + tid * zld;
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
      for (int i = 0; i + 1 < N; ++i) {
        const float c = gk[i];
        const float nd = -lmb;
        const float ns = (i + 2 < N) ? gk[i + 1] : 0.f;
        const float yn = (it == 0) ? start(i + 1) : y[i + 1] * inv;
        const bool piv = fabsf(a) >= fabsf(c);
        const float den = piv ? ((a == 0.f) ? tp : a) : c;
        const float rd = 1.f / den;
        const float mlt = (piv ? c : a) * rd;
        const float yo = piv ? yk : yn, ye = piv ? yn : yk;
        u2[i] = (piv ? bb : nd) * rd;
        u3[i] = piv ? 0.f : ns * rd;
        y[i] = yo * rd;
        yk = fmaf(-mlt, yo, ye);
        a = piv ? fmaf(-mlt, bb, nd) : fmaf(-mlt, nd, bb);
        bb = piv ? ns : -mlt * ns;
      }
      if (a == 0.f) a = tp;
      float x2 = yk / a;
      y[N - 1] = x2;
      float x1 = x2;
      float mx = fabsf(x2);
      if (N >= 2) {
        x1 = fmaf(-u2[N - 2], x2, y[N - 2]);
        y[N - 2] = x1;
        mx = fmaxf(mx, fabsf(x1));
      }
      for (int i = N - 3; i >= 0; --i) {
        const float xi = y[i] - u2[i] * x1 - u3[i] * x2;
        y[i] = xi;
        mx = fmaxf(mx, fabsf(xi));
        x2 = x1;
        x1 = xi;
      }
      inv = (mx > 0.f && isfinite(mx)) ? 1.f / mx : 1.f;
    }
    shift[tid] = inv;  // read back as the vector's scale
  }
  __syncthreads();

  // ---- d. vectors: thread quad (column col, quarter qr) holds rows
  // kk * 4 + qr of its vector: the odd entries of the T_GK vector
  const int col = tid >> 2, qr = tid & 3;
  const bool live = col < r;
  float z[kQ];
  {
    const float vs = live ? shift[col] : 0.f;
#pragma unroll
    for (int kk = 0; kk < kQ; ++kk) {
      const int row = kk * 4 + qr;
      z[kk] = (live && row < p) ? Zs[col * zld + 2 * row + 1] * vs : 0.f;
    }
  }
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
  __syncthreads();  // Zs reads done before pub writes (pub is separate, but keep order simple)
  auto normalise_publish = [&](float* dst) {
    const float s = quad_sum(dot32(z, z));
    const float iv = (s > 0.f) ? 1.f / sqrtf(s) : 0.f;
#pragma unroll
    for (int kk = 0; kk < kQ; ++kk) {
      z[kk] *= iv;
      dst[kk * 4 + qr] = z[kk];
    }
  };
  if (col == 0) normalise_publish(pub);
  for (int j = 0; j < r; ++j) {
    __syncthreads();  // vector j published; reads of the other buffer done
    if (live && col > j) {
      const float* pv = pub + (j & 1) * 132;
      float pj[kQ];
#pragma unroll
      for (int kk = 0; kk < kQ; ++kk) pj[kk] = pv[kk * 4 + qr];
      const float d = quad_sum(dot32(pj, z));
#pragma unroll
      for (int kk = 0; kk < kQ; ++kk) z[kk] = fmaf(-d, pj[kk], z[kk]);
      if (col == j + 1) normalise_publish(pub + ((j + 1) & 1) * 132);
    }
  }
  if (live) {
    // U = H_0 ... H_{p-1} [u; 0]: reflector k covers rows k .. m-1 with
    // entry 1 at row k and the packed entries below
    for (int k = p - 1; k >= 0; --k) {
      const float tk = tau[k];
      if (tk == 0.f) continue;
      const int ro = refl_off(k, m);
      float vk[kQ];
#pragma unroll
      for (int kk = 0; kk < kQ; ++kk) {
        const int row = kk * 4 + qr;
        vk[kk] = (row == k) ? 1.f : ((row > k && row < m) ? Refl[ro + row - k - 1] : 0.f);
      }
      const float d = quad_sum(dot32(vk, z)) * tk;
#pragma unroll
      for (int kk = 0; kk < kQ; ++kk) z[kk] = fmaf(-d, vk[kk], z[kk]);
    }
    float best = -1.f;
    int bi = kNmax;
#pragma unroll
    for (int kk = 0; kk < kQ; ++kk) {
      const int row = kk * 4 + qr;
      const float a = fabsf(z[kk]);
      if (row < m && (a > best || (a == best && row < bi))) { best = a; bi = row; }
    }
    const unsigned qm = 0xFu << (threadIdx.x & 28);
    for (int o = 1; o <= 2; o <<= 1) {
      const float ob = __shfl_xor_sync(qm, best, o);
      const int oi = __shfl_xor_sync(qm, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    float sv = 0.f;
#pragma unroll
    for (int kk = 0; kk < kQ; ++kk)
      if (kk * 4 + qr == bi) sv = z[kk];
    sv = quad_sum(sv);
    const float sg = (sv < 0.f) ? -1.f : 1.f;
    float* U = Ug + (long long)b * sU;
    float* Ut = Utg ? Utg + (long long)b * sUt + (long long)col * m : nullptr;
#pragma unroll
    for (int kk = 0; kk < kQ; ++kk) {
      const int row = kk * 4 + qr;
      if (row < m) {
        U[(long long)row * r + col] = sg * z[kk];
        if (Ut) Ut[row] = sg * z[kk];
      }
    }
  }
  if (lamg) {
    double* lo = lamg + (long long)b * slam;
    for (int t = tid; t < nlam; t += kThreads) {
      const double s = (t < nl) ? double(lam[t]) : 0.0;
      lo[t] = s * s;
    }
  }
}

}  // namespace

size_t chol_env_smem_bytes(int n) { return sizeof(float) * (size_t(n) * (n | 1) + n); }

cudaError_t launch_chol_env(float* R, long long sR, const int64_t* r_off, const int32_t* D,
                            int maxD, const unsigned int* amax, long long s_amax, int k0, int nk,
                            int batch, cudaStream_t st) {
  if (maxD < 1 || maxD > kNmax || nk < 1) return cudaErrorInvalidValue;
  const size_t smem = chol_env_smem_bytes(maxD);
  k_chol_env<<<batch * nk, kThreads, smem, st>>>(R, sR, r_off, D, amax, s_amax, k0, nk);
  return cudaGetLastError();
}

size_t svd_left_smem_bytes(int m, int n, int r) {
  const SvdLayout L = svd_layout(m, n, r);
  return sizeof(float) * (size_t(L.region) + size_t(L.refl) + size_t(kSmallFloats));
}

bool svd_left_supported(int m, int n, int r) {
  return m >= 1 && n >= 1 && m <= kNmax && n <= kNmax && r >= 1 && r <= kRmax &&
         r <= (m < n ? m : n);
}

cudaError_t launch_svd_left(const float* K, long long sK, int m, int n, float* U, long long sU,
                            float* Ut, long long sUt, double* lam, long long slam, int r,
                            int nlam, int* status, int batch, cudaStream_t st) {
  if (!svd_left_supported(m, n, r) || nlam < 0 || nlam > m) return cudaErrorInvalidValue;
  const size_t smem = svd_left_smem_bytes(m, n, r);
  k_svd_left<<<batch, kThreads, smem, st>>>(K, sK, m, n, U, sU, Ut, sUt, lam, slam, r, nlam,
                                            status);
  return cudaGetLastError();
}

cudaError_t svd_configure() {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  const size_t need_svd = svd_left_smem_bytes(kNmax, kNmax, kRmax);
  const size_t need_chol = chol_env_smem_bytes(kNmax);
  if (need_svd > size_t(optin) || need_chol > size_t(optin)) return cudaErrorInvalidValue;
  e = cudaFuncSetAttribute(k_svd_left, cudaFuncAttributeMaxDynamicSharedMemorySize, int(need_svd));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_chol_env, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              int(need_chol));
}

}  // namespace tn
