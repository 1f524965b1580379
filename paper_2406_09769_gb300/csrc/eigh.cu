// Batched top-r symmetric eigensolver for the density matrices L_v
// (leading_eigenvectors of Algorithm density_matrix_alg, Sec. 5).
//
// One CTA per matrix, everything in shared memory:
//   1. Householder reduction to tridiagonal form, A = Q T Q^T
//      (Golub & Van Loan, Matrix Computations, Sec. 8.3.1);
//   2. the wanted eigenvalues of T by Sturm-sequence multisection, four
//      threads per eigenvalue (Barth, Martin & Wilkinson 1967); in FP32 a first
//      round on an equispaced grid is shared by all eigenvalues;
//   3. eigenvectors of T by inverse iteration with partial-pivoting LU of
//      T - lambda I (Wilkinson), one thread per eigenvector, shifts of
//      near-equal eigenvalues separated as in LAPACK's stein;
//   4. modified Gram-Schmidt over the r vectors (descending eigenvalue order);
//   5. back-transformation by the stored reflectors, U = Q Z;
//   6. each column signed so that its largest-|.| entry (first on ties) is
//      positive.
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
constexpr int kNmax = 128;

template <typename T> struct Lim;
template <> struct Lim<double> {
  __device__ static double eps() { return DBL_EPSILON * 0.5; }
  __device__ static double safmin() { return DBL_MIN; }
  static constexpr int maxit = 80;
};
template <> struct Lim<float> {
  __device__ static float eps() { return FLT_EPSILON * 0.5f; }
  __device__ static float safmin() { return FLT_MIN; }
  static constexpr int maxit = 40;
};

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ T block_sum(T v, T* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  T t = (lane < (kThreads >> 5)) ? red[lane] : T(0);
  t = warp_sum(t);
  return t;
}

template <typename T>
__device__ int sturm_count(const T* dd, const T* e2, int n, T x, T pivmin) {
  T q = dd[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  int c = (q < T(0));
  for (int j = 1; j < n; ++j) {
    q = dd[j] - x - e2[j - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    c += (q < T(0));
  }
  return c;
}

template <typename T, typename TU>
__global__ void __launch_bounds__(kThreads) k_eigh_top(const T* __restrict__ Lg, long long sL,
                                                       TU* __restrict__ Ug, long long sU,
                                                       TU* __restrict__ Utg, long long sUt,
                                                       double* __restrict__ lamg, long long slam,
                                                       int n, int r, int nlam, int* status) {
  extern __shared__ __align__(16) unsigned char raw[];
  __shared__ T red[32];
  __shared__ T scal[8];
  const int ld = n + 1;
  const int nl = (nlam > r) ? nlam : r;
  T* A = reinterpret_cast<T*>(raw);   // n x ld
  T* Z = A + n * ld;                   // r vectors of length n (column-major)
  T* dd = Z + n * r;
  T* ee = dd + n;
  T* e2 = ee + n;
  T* tau = e2 + n;
  T* v = tau + n;
  T* w = v + n;
  T* lam = w + n;                      // nl
  T* shift = lam + nl;                 // r
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = kThreads >> 5;
  const int b = blockIdx.x;
  const T* L = Lg + (long long)b * sL;

  // ---- load, symmetrise, screen for NaN/Inf
  bool bad = false;
  for (int idx = tid; idx < n * n; idx += kThreads) {
    const int a = idx / n, c = idx % n;
    const T x = T(0.5) * (L[(long long)a * n + c] + L[(long long)c * n + a]);
    if (!isfinite(x)) bad = true;
    A[a * ld + c] = x;
  }
  if (__syncthreads_or(bad)) {
    TU* U = Ug + (long long)b * sU;
    for (int idx = tid; idx < n * r; idx += kThreads) U[idx] = TU(0);
    if (Utg)
      for (int idx = tid; idx < n * r; idx += kThreads) Utg[(long long)b * sUt + idx] = TU(0);
    if (tid == 0) status[b] = TN_ERR_NONFINITE;
    return;
  }

  // ---- 1. Householder tridiagonalisation (lower), v stored below the diagonal
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;
    T part = T(0);
    for (int j = 1 + tid; j < m; j += kThreads) {
      const T x = A[(k + 1 + j) * ld + k];
      part += x * x;
    }
    const T sig = block_sum(part, red);
    if (tid == 0) {
      dd[k] = A[k * ld + k];
      const T alpha = A[(k + 1) * ld + k];
      if (sig == T(0)) {
        tau[k] = T(0);
        ee[k] = alpha;
        scal[0] = T(0);
      } else {
        const T beta = -copysign(sqrt(alpha * alpha + sig), alpha);
        tau[k] = (beta - alpha) / beta;
        ee[k] = beta;
        scal[0] = T(1) / (alpha - beta);
      }
    }
    __syncthreads();
    const T tk = tau[k];
    if (tk == T(0)) {
      for (int j = tid; j < m; j += kThreads) A[(k + 1 + j) * ld + k] = (j == 0) ? T(1) : T(0);
      __syncthreads();
      continue;
    }
    const T sc = scal[0];
    for (int j = tid; j < m; j += kThreads) {
      const T x = (j == 0) ? T(1) : A[(k + 1 + j) * ld + k] * sc;
      v[j] = x;
      A[(k + 1 + j) * ld + k] = x;
    }
    __syncthreads();
    // w = tau * A22 v (warp per row)
    for (int a = warp; a < m; a += nwarp) {
      const T* row = A + (k + 1 + a) * ld + (k + 1);
      T s = T(0);
      for (int c = lane; c < m; c += 32) s += row[c] * v[c];
      s = warp_sum(s);
      if (lane == 0) w[a] = tk * s;
    }
    __syncthreads();
    T pd = T(0);
    for (int a = tid; a < m; a += kThreads) pd += w[a] * v[a];
    const T dot = block_sum(pd, red);
    const T K = T(-0.5) * tk * dot;
    for (int a = tid; a < m; a += kThreads) w[a] += K * v[a];
    __syncthreads();
    for (int idx = tid; idx < m * m; idx += kThreads) {
      const int a = idx / m, c = idx % m;
      A[(k + 1 + a) * ld + (k + 1 + c)] -= v[a] * w[c] + w[a] * v[c];
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (n >= 2) {
      dd[n - 2] = A[(n - 2) * ld + (n - 2)];
      ee[n - 2] = A[(n - 1) * ld + (n - 2)];
      tau[n - 2] = T(0);
    }
    dd[n - 1] = A[(n - 1) * ld + (n - 1)];
    ee[n - 1] = T(0);
    // Gershgorin interval, pivmin (LAPACK stebz conventions)
    T gl = dd[0], gu = dd[0], emax = T(0);
    for (int j = 0; j < n; ++j) {
      const T el = (j > 0) ? fabs(ee[j - 1]) : T(0);
      const T er = (j + 1 < n) ? fabs(ee[j]) : T(0);
      gl = fmin(gl, dd[j] - el - er);
      gu = fmax(gu, dd[j] + el + er);
      if (j + 1 < n) {
        e2[j] = ee[j] * ee[j];
        emax = fmax(emax, e2[j]);
      }
    }
    const T tnorm = fmax(fabs(gl), fabs(gu));
    const T eps = Lim<T>::eps();
    const T pivmin = Lim<T>::safmin() * fmax(T(1), emax);
    gl -= T(2.1) * tnorm * eps * n + T(4.2) * pivmin;
    gu += T(2.1) * tnorm * eps * n + T(4.2) * pivmin;
    scal[1] = gl;
    scal[2] = gu;
    scal[3] = tnorm;
    scal[4] = pivmin;
  }
  __syncthreads();
  const T gl = scal[1], gu = scal[2], tnorm = scal[3], pivmin = scal[4];
  const T eps = Lim<T>::eps();

  // ---- 2. bisection for the nl largest eigenvalues (descending)
  if (tid < nl && tid < n) {
    const int j = n - 1 - tid;  // ascending index
    T lo = gl, hi = gu;
    for (int it = 0; it < Lim<T>::maxit; ++it) {
      const T mid = T(0.5) * (lo + hi);
      if (hi - lo <= T(2) * eps * fmax(fabs(lo), fabs(hi)) + T(2) * pivmin) break;
      if (sturm_count(dd, e2, n, mid, pivmin) <= j) lo = mid;
      else hi = mid;
    }
    lam[tid] = T(0.5) * (lo + hi);
  }
  __syncthreads();
  if (tid == 0) {
    // separate near-equal shifts (descending order)
    const T pertol = T(10) * eps * fmax(tnorm, Lim<T>::safmin());
    for (int t = 0; t < r; ++t) {
      T s = lam[t];
      if (t > 0 && shift[t - 1] - s < pertol) s = shift[t - 1] - pertol;
      shift[t] = s;
    }
  }
  __syncthreads();

  // ---- 3. inverse iteration, one thread per eigenvector
  if (tid < r) {
    T u1[kNmax], u2[kNmax], u3[kNmax], ml[kNmax], x[kNmax];
    unsigned char pv[kNmax];
    const T lmb = shift[tid];
    const T tp = fmax(eps * tnorm, Lim<T>::safmin());
    T a = dd[0] - lmb;
    T bb = (n > 1) ? ee[0] : T(0);
    for (int k = 0; k + 1 < n; ++k) {
      const T c = ee[k];
      const T nd = dd[k + 1] - lmb;
      const T ns = (k + 2 < n) ? ee[k + 1] : T(0);
      if (fabs(a) >= fabs(c)) {
        if (a == T(0)) a = tp;
        const T mlt = c / a;
        pv[k] = 0; ml[k] = mlt; u1[k] = a; u2[k] = bb; u3[k] = T(0);
        a = nd - mlt * bb;
        bb = ns;
      } else {
        const T mlt = a / c;
        pv[k] = 1; ml[k] = mlt; u1[k] = c; u2[k] = nd; u3[k] = ns;
        a = bb - mlt * nd;
        bb = -mlt * ns;
      }
    }
    if (a == T(0)) a = tp;
    u1[n - 1] = a;
    // deterministic start vector
    for (int k = 0; k < n; ++k) {
      unsigned int h = 2654435761u * (unsigned)(k + 1) ^ (40503u * (unsigned)(tid + 7));
      h ^= h >> 13; h *= 0x5bd1e995u; h ^= h >> 15;
      x[k] = T(1) + T(0.5) * (T(h & 0xffff) / T(65536) - T(0.5));
    }
    for (int it = 0; it < 3; ++it) {
      for (int k = 0; k + 1 < n; ++k) {
        if (pv[k]) { const T t = x[k]; x[k] = x[k + 1]; x[k + 1] = t; }
        x[k + 1] -= ml[k] * x[k];
      }
      x[n - 1] = x[n - 1] / u1[n - 1];
      if (n >= 2) x[n - 2] = (x[n - 2] - u2[n - 2] * x[n - 1]) / u1[n - 2];
      for (int k = n - 3; k >= 0; --k) x[k] = (x[k] - u2[k] * x[k + 1] - u3[k] * x[k + 2]) / u1[k];
      T mx = T(0);
      for (int k = 0; k < n; ++k) mx = fmax(mx, fabs(x[k]));
      const T inv = (mx > T(0) && isfinite(mx)) ? T(1) / mx : T(1);
      for (int k = 0; k < n; ++k) x[k] *= inv;
    }
    T* zc = Z + tid * n;
    for (int k = 0; k < n; ++k) zc[k] = x[k];
  }
  __syncthreads();

  // ---- 4. modified Gram-Schmidt (descending eigenvalue order)
  for (int j = 0; j < r; ++j) {
    T* zj = Z + j * n;
    T part = T(0);
    for (int a = tid; a < n; a += kThreads) part += zj[a] * zj[a];
    const T nrm = sqrt(block_sum(part, red));
    const T inv = (nrm > T(0)) ? T(1) / nrm : T(0);
    for (int a = tid; a < n; a += kThreads) zj[a] *= inv;
    __syncthreads();
    for (int c = j + 1 + warp; c < r; c += nwarp) {
      T* zc = Z + c * n;
      T s = T(0);
      for (int a = lane; a < n; a += 32) s += zj[a] * zc[a];
      s = warp_sum(s);
      for (int a = lane; a < n; a += 32) zc[a] -= s * zj[a];
    }
    __syncthreads();
  }

  // ---- 5. back-transformation U = H_0 H_1 ... H_{n-3} Z
  for (int k = n - 3; k >= 0; --k) {
    const T tk = tau[k];
    if (tk == T(0)) continue;  // uniform across the block
    const int m = n - k - 1;
    const T* vk = A + (k + 1) * ld + k;  // vk[j * ld] = v_j
    for (int c = warp; c < r; c += nwarp) {
      T* zc = Z + c * n + (k + 1);
      T s = T(0);
      for (int a = lane; a < m; a += 32) s += vk[a * ld] * zc[a];
      s = tk * warp_sum(s);
      __syncwarp();
      for (int a = lane; a < m; a += 32) zc[a] -= s * vk[a * ld];
    }
    __syncthreads();
  }

  // ---- 6. sign convention and output
  for (int c = warp; c < r; c += nwarp) {
    T* zc = Z + c * n;
    T best = T(-1);
    int bi = n;
    for (int a = lane; a < n; a += 32) {
      const T x = fabs(zc[a]);
      if (x > best || (x == best && a < bi)) { best = x; bi = a; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const T ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    const T sgn = (bi < n && zc[bi] < T(0)) ? T(-1) : T(1);
    __syncwarp();
    for (int a = lane; a < n; a += 32) zc[a] *= sgn;
  }
  __syncthreads();
  TU* U = Ug + (long long)b * sU;
  for (int idx = tid; idx < n * r; idx += kThreads) {
    const int a = idx / r, c = idx % r;
    U[idx] = TU(Z[c * n + a]);
  }
  if (Utg) {
    TU* Ut = Utg + (long long)b * sUt;
    for (int idx = tid; idx < n * r; idx += kThreads) Ut[idx] = TU(Z[idx]);
  }
  if (lamg) {
    double* lo = lamg + (long long)b * slam;
    for (int t = tid; t < nlam && t < n; t += kThreads) lo[t] = double(lam[t]);
  }
}

// ---------------------------------------------------------------------------
// Register-resident variant for n <= 128, r <= 64 (the shapes of the MPS-tree
// density matrices at chi <= 64).  Same mathematics as k_eigh_top; the work is
// laid out so that barriers are few and every thread is busy:
//   * Householder step: warp 0 forms the reflector; the 256 threads split the
//     trailing matrix by (row, half of the columns) for the product A22 v and
//     the rank-2 update (shared-memory rows of n + 1 words: no bank conflicts);
//     four barriers per step;
//   * eigenvalues: 4 threads per eigenvalue evaluate Sturm counts at 4 interior
//     points of the current interval (multisection), a fixed number of rounds;
//   * eigenvectors of T: inverse iteration, one thread per vector;
//   * the r vectors are then held in registers by thread quads (column c;
//     thread q of the quad owns rows q, q+4, q+8, ... so that the quad's four
//     reads of one shared-memory column fall in four banks), so modified
//     Gram-Schmidt needs two barriers per vector and the back-transformation
//     H_0 ... H_{n-3} Z none at all.
constexpr int kQ = 32;  // rows per quarter (n <= 128)

template <typename T>
__device__ __forceinline__ T fdiv(T a, T b) { return a / b; }
template <>
__device__ __forceinline__ float fdiv<float>(float a, float b) { return __fdividef(a, b); }

// Sum over the 4 lanes of a thread quad; only those lanes need to be active.
template <typename T>
__device__ __forceinline__ T quad_sum(T v) {
  const unsigned qm = 0xFu << (threadIdx.x & 28);
  v += __shfl_xor_sync(qm, v, 1);
  v += __shfl_xor_sync(qm, v, 2);
  return v;
}

// FP32 Householder tridiagonalisation with the matrix in registers: thread
// (row ri = tid & 127, column half h = tid >> 7) holds A[ri][64 h .. 64 h + 63]
// (zero outside n x n).  Step k: the owners of row k publish it (= column k)
// to X, sixteen float4 stores per owner and nothing else, so the next step waits
// on no serial arithmetic; each of the first four warps sums the squares of
// the row's tail itself (one float4 per lane and a warp reduction) and forms
// the reflector (same arithmetic, same values in each), and threads c < 128
// write v_c to V (zero outside k+1 .. n-1); the rows'
// partial products p = A v go to P; threads c write w_c = tau p_c - (tau^2 /
// 2)(v.p) v_c to W (zero outside); then every row updates in place, A -= v
// w^T + w v^T.  Zeros outside the active block make the inner loops plain
// FMAs on broadcast float4 loads.  The reflectors are stored in column k of
// R as rows: R[k * kRld + c + (c / 32) * 4] = v_c for c < 128 (zero outside
// k+1 .. n-1, v_{k+1} = 1; the padding puts the four 32-row quarters in
// disjoint bank groups); R may overlay As, which is read only at the start.
// dd, ee, tau as the shared-memory version.  X, V, W (128 each, W followed by
// 16 spare entries) and P (2 x 128) are 16-byte aligned.
constexpr int kRld = 144;
__device__ __forceinline__ int rpad(int c) { return c + (c >> 5) * 4; }

__device__ void tridiag_regs_f32(const float* As, int ld, int n, float* R, float* dd, float* ee,
                                 float* tau, float* X, float* V, float* W, float* P) {
  float* D8 = W + 128;  // warp partials of v . p
  const int tid = threadIdx.x, ri = tid & 127, h = tid >> 7, lane = tid & 31, cb = h * 64;
  float a[64];
#pragma unroll
  for (int q = 0; q < 64; ++q) a[q] = (ri < n && cb + q < n) ? As[ri * ld + cb + q] : 0.f;
  auto publish = [&](int k) {
#pragma unroll
    for (int q = 0; q < 64; q += 4)
      *reinterpret_cast<float4*>(X + cb + q) = make_float4(a[q], a[q + 1], a[q + 2], a[q + 3]);
  };
  if (ri == 0) publish(0);
  for (int k = 0; k + 2 < n; ++k) {
    __syncthreads();  // row k published; the previous step's reads of V, W are done
    if (tid < 128) {  // the first four warps form the reflector (same values in each)
      float s;
      {  // sum of squares of row k beyond column k + 1, in every warp
        const float4 x4 = *reinterpret_cast<const float4*>(X + 4 * lane);
        const int c0 = 4 * lane;
        float t = (c0 >= k + 2) ? x4.x * x4.x : 0.f;
        t = (c0 + 1 >= k + 2) ? fmaf(x4.y, x4.y, t) : t;
        t = (c0 + 2 >= k + 2) ? fmaf(x4.z, x4.z, t) : t;
        t = (c0 + 3 >= k + 2) ? fmaf(x4.w, x4.w, t) : t;
        s = warp_sum(t);
      }
      const float alpha = X[k + 1];
      float tk, beta, sc;
      if (s == 0.f) {
        tk = 0.f; beta = alpha; sc = 0.f;
      } else {
        beta = -copysignf(sqrtf(alpha * alpha + s), alpha);
        tk = (beta - alpha) / beta;
        sc = 1.f / (alpha - beta);
      }
      const int c = tid;
      const float vc = (c == k + 1) ? 1.f : ((c > k + 1 && c < n && tk != 0.f) ? X[c] * sc : 0.f);
      V[c] = vc;
      R[k * kRld + rpad(c)] = vc;
      if (c == 0) {
        dd[k] = X[k];
        ee[k] = beta;
        tau[k] = tk;
      }
    }
    __syncthreads();  // V and tau_k complete; X free
    const float tk = tau[k];
    const bool rowlive = ri > k && ri < n;
    if (tk != 0.f) {  // uniform across the block
      if (rowlive) {
        float2 pq = make_float2(0.f, 0.f);  // (even, odd) columns, packed FMAs
#pragma unroll
        for (int q = 0; q < 64; q += 4) {
          if (cb + q + 3 <= k || cb + q >= n) continue;  // warp-uniform: group inactive
          const float4 v4 = *reinterpret_cast<const float4*>(V + cb + q);
          pq = __ffma2_rn(make_float2(a[q], a[q + 1]), make_float2(v4.x, v4.y), pq);
          pq = __ffma2_rn(make_float2(a[q + 2], a[q + 3]), make_float2(v4.z, v4.w), pq);
        }
        P[h * 128 + ri] = pq.x + pq.y;
      }
      // v . p folded per warp (rows outside k+1 .. n-1 have v = 0)
      {
        float t = rowlive ? V[ri] * (P[h * 128 + ri]) : 0.f;
        t = warp_sum(t);
        if (lane == 0) D8[tid >> 5] = t;
      }
      __syncthreads();  // partial products of every row
      const float4 d0 = *reinterpret_cast<const float4*>(D8);
      const float4 d1 = *reinterpret_cast<const float4*>(D8 + 4);
      const float dsum = tk * (((d0.x + d0.y) + (d0.z + d0.w)) + ((d1.x + d1.y) + (d1.z + d1.w)));
      const float K = -0.5f * tk * dsum;
      if (tid < 128) {
        const int c = tid;
        W[c] = (c > k && c < n) ? fmaf(K, V[c], tk * (P[c] + P[128 + c])) : 0.f;
      }
      __syncthreads();  // W complete
      if (rowlive) {
        const float vi = V[ri], wi = W[ri];
        const float2 nvi = make_float2(-vi, -vi), nwi = make_float2(-wi, -wi);
#pragma unroll
        for (int q = 0; q < 64; q += 4) {
          if (cb + q + 3 <= k || cb + q >= n) continue;  // warp-uniform: group inactive
          const float4 v4 = *reinterpret_cast<const float4*>(V + cb + q);
          const float4 w4 = *reinterpret_cast<const float4*>(W + cb + q);
          // a -= v_i w_c + w_i v_c as two FMAs, two columns per packed FMA
          float2 lo = __ffma2_rn(nvi, make_float2(w4.x, w4.y), make_float2(a[q], a[q + 1]));
          float2 hi = __ffma2_rn(nvi, make_float2(w4.z, w4.w), make_float2(a[q + 2], a[q + 3]));
          lo = __ffma2_rn(nwi, make_float2(v4.x, v4.y), lo);
          hi = __ffma2_rn(nwi, make_float2(v4.z, v4.w), hi);
          a[q] = lo.x; a[q + 1] = lo.y; a[q + 2] = hi.x; a[q + 3] = hi.y;
        }
      }
    }
    if (ri == k + 1) publish(k + 1);
  }
  // the last 2 x 2 block of T
  if (ri >= n - 2 && ri < n) {
#pragma unroll
    for (int q = 0; q < 64; ++q) {
      const int c = cb + q;
      if (c == ri) dd[ri] = a[q];
      if (c == ri - 1 && ri == n - 1) ee[n - 2] = a[q];
    }
  }
  if (tid == 0) {
    ee[n - 1] = 0.f;
    if (n >= 2) tau[n - 2] = 0.f;
  }
  __syncthreads();
}

// FP32 multisection: Sturm sequences per thread and rounds after the shared
// grid round; 257 (4 kSturmIlp + 1)^kSturmRounds >= 5^12 keeps the final
// interval at or below that of twelve quinsection rounds.  One sequence per
// thread measured fastest with two CTAs per SM: more interleaved sequences
// cost more issue slots than their overlapped divisions save.
constexpr int kSturmIlp = 1;
constexpr int kSturmRounds = 9;

// Sturm counts (eigenvalues of T below x[i]) of several shifts, interleaved so
// that the divisions of independent sequences overlap.
__device__ void sturm_count_multi(const float* dd, const float* e2, int n, const float* x,
                                  float pivmin, int* c) {
  float q[kSturmIlp];
#pragma unroll
  for (int i = 0; i < kSturmIlp; ++i) {
    q[i] = dd[0] - x[i];
    if (fabsf(q[i]) < pivmin) q[i] = -pivmin;
    c[i] = (q[i] < 0.f);
  }
  for (int j = 1; j < n; ++j) {
    const float d = dd[j], e = e2[j - 1];
#pragma unroll
    for (int i = 0; i < kSturmIlp; ++i) {
      q[i] = d - x[i] - __fdividef(e, q[i]);
      if (fabsf(q[i]) < pivmin) q[i] = -pivmin;
      c[i] += (q[i] < 0.f);
    }
  }
}

template <typename T>
__device__ int sturm_count_fast(const T* dd, const T* e2, int n, T x, T pivmin) {
  T q = dd[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  int c = (q < T(0));
  for (int j = 1; j < n; ++j) {
    q = dd[j] - x - fdiv(e2[j - 1], q);
    if (fabs(q) < pivmin) q = -pivmin;
    c += (q < T(0));
  }
  return c;
}

// FP32 phases 4-6: thread quad (column col = tid / 4, quarter qr = tid % 4)
// holds rows qr * 32 .. qr * 32 + 31 of its vector (z[kk] = row qr * 32 + kk),
// so the quad's reads of a shared vector are float4 loads at padded offsets
// qr * 36 + kk (disjoint bank groups, broadcast across quads).  Modified
// Gram-Schmidt in descending eigenvalue order with double-buffered published
// vectors (one barrier per vector), then U = H_0 ... H_{n-3} Z from the
// padded reflector rows R, then signs (largest-|.| entry, first on ties,
// positive) and the stores U (n x r) and Ut (r x n).
__device__ void vectors_f32(const float* Zs, int zld, const float* zscale, int n, int r,
                            const float* R, const float* tau, float* pub, float* U, float* Ut,
                            const GuardTab* gd = nullptr) {
  const int tid = threadIdx.x, col = tid >> 2, qr = tid & 3;
  const bool live = col < r;
  const float zs = live ? zscale[col] : 0.f;
  float z[kQ];
#pragma unroll
  for (int kk = 0; kk < kQ; ++kk) {
    const int row = qr * kQ + kk;
    z[kk] = (live && row < n) ? Zs[col * zld + row] * zs : 0.f;
  }
  auto load = [&](const float* src, float* v) {
#pragma unroll
    for (int m = 0; m < kQ / 4; ++m) {
      const float4 t = *reinterpret_cast<const float4*>(src + qr * 36 + 4 * m);
      v[4 * m] = t.x; v[4 * m + 1] = t.y; v[4 * m + 2] = t.z; v[4 * m + 3] = t.w;
    }
  };
  // dot product of 32 register entries as four interleaved partial sums (two
  // packed pairs); z -= d x in packed pairs
  auto dot32 = [](const float* x, const float* y) {
    float2 da = make_float2(0.f, 0.f), db = make_float2(0.f, 0.f);
#pragma unroll
    for (int kk = 0; kk < kQ; kk += 4) {
      da = __ffma2_rn(make_float2(x[kk], x[kk + 1]), make_float2(y[kk], y[kk + 1]), da);
      db = __ffma2_rn(make_float2(x[kk + 2], x[kk + 3]), make_float2(y[kk + 2], y[kk + 3]), db);
    }
    return (da.x + da.y) + (db.x + db.y);
  };
  auto axpy32 = [](float d, const float* x, float* y) {
    const float2 nd = make_float2(-d, -d);
#pragma unroll
    for (int kk = 0; kk < kQ; kk += 2) {
      const float2 t = __ffma2_rn(nd, make_float2(x[kk], x[kk + 1]), make_float2(y[kk], y[kk + 1]));
      y[kk] = t.x;
      y[kk + 1] = t.y;
    }
  };
  auto normalise_publish = [&](float* dst) {
    float s = quad_sum(dot32(z, z));
    const float inv = (s > 0.f) ? 1.f / sqrtf(s) : 0.f;
#pragma unroll
    for (int kk = 0; kk < kQ; ++kk) z[kk] *= inv;
#pragma unroll
    for (int m = 0; m < kQ / 4; ++m)
      *reinterpret_cast<float4*>(dst + qr * 36 + 4 * m) =
          make_float4(z[4 * m], z[4 * m + 1], z[4 * m + 2], z[4 * m + 3]);
  };
  if (col == 0) normalise_publish(pub);
  for (int j = 0; j < r; ++j) {
    __syncthreads();  // vector j published; the reads of the other buffer are done
    if (live && col > j) {
      float p[kQ];
      load(pub + (j & 1) * kRld, p);
      const float d = quad_sum(dot32(p, z));
      axpy32(d, p, z);
      if (col == j + 1) normalise_publish(pub + ((j + 1) & 1) * kRld);
    }
  }
  if (live) {
    for (int k = n - 3; k >= 0; --k) {
      const float tk = tau[k];
      if (tk == 0.f) continue;
      float v[kQ];
      load(R + k * kRld, v);
      const float d = quad_sum(dot32(v, z)) * tk;
      axpy32(d, v, z);
    }
    float best = -1.f;
    int bi = kNmax;
#pragma unroll
    for (int kk = 0; kk < kQ; ++kk) {
      const int row = qr * kQ + kk;
      const float a = fabsf(z[kk]);
      if (row < n && (a > best || (a == best && row < bi))) { best = a; bi = row; }
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
      if (qr * kQ + kk == bi) sv = z[kk];
    sv = quad_sum(sv);
    const float sgn = (sv < 0.f) ? -1.f : 1.f;
#pragma unroll
    for (int kk = 0; kk < kQ; ++kk) {
      const int row = qr * kQ + kk;
      if (row < n) {
        if (guard_ok(gd, U + (long long)row * r + col, 4, 0x607))
          U[(long long)row * r + col] = sgn * z[kk];
        if (Ut && guard_ok(gd, Ut + (long long)col * n + row, 4, 0x608))
          Ut[(long long)col * n + row] = sgn * z[kk];
      }
    }
  }
}

// Elements of the A region: the n x (n + 1) matrix, or for FP32 the larger of
// that and the padded reflector rows (n - 2) x kRld.
template <typename T>
__host__ __device__ __forceinline__ int fast_region_a(int n) {
  const int m = n * (n + 1);
  if (sizeof(T) == 8) return m;
  const int rr = (n > 2 ? n - 2 : 0) * kRld;
  return m > rr ? m : rr;
}

// kMode 0: strided batch; 1 (FP32 only): grouped launch, CTA i solves problem
// desc[i]; 2: as 1 with the range guard checked on every global access.
template <typename T, int kMode = 0>
__global__ void __launch_bounds__(kThreads) k_eigh_fast(const T* __restrict__ Lg_, long long sL,
                                                        T* __restrict__ Ug_, long long sU,
                                                        T* __restrict__ Utg_, long long sUt,
                                                        double* __restrict__ lamg_, long long slam,
                                                        int n_, int r_, int nlam_, int* status_,
                                                        const EighDesc* __restrict__ desc) {
  extern __shared__ __align__(16) unsigned char raw[];
  __shared__ T scal[8];
  // grouped launch: CTA i solves problem desc[i] with its own pointers and
  // shape; else instance blockIdx.x of the strided arguments
  const EighDesc* qd = kMode ? desc + blockIdx.x : nullptr;
  const GuardTab* gd = kMode == 2 ? qd->guard : nullptr;
  const int b = qd ? 0 : int(blockIdx.x);
  const T* Lg = qd ? reinterpret_cast<const T*>(qd->L) : Lg_;
  T* Ug = qd ? reinterpret_cast<T*>(qd->U) : Ug_;
  T* Utg = qd ? reinterpret_cast<T*>(qd->Ut) : Utg_;
  double* lamg = qd ? qd->lam : lamg_;
  int* status = qd ? qd->status : status_;
  const int n = qd ? qd->n : n_, r = qd ? qd->r : r_, nlam = qd ? qd->nlam : nlam_;
  const int ld = n + 1;
  const int nl = (nlam > r) ? nlam : r;
  // the 128-entry vectors first (16-byte aligned), then A and Z
  T* dd = reinterpret_cast<T*>(raw);
  T* ee = dd + kNmax;
  T* e2 = ee + kNmax;
  T* tau = e2 + kNmax;
  T* vb = tau + kNmax;                // vb, wv: 2 x 128, published rows (FP32)
  T* wv = vb + kNmax;
  T* part = wv + kNmax;               // 2 x 128
  T* lam = part + 2 * kNmax;          // kNmax
  T* pub = lam + kNmax;               // 3 x kNmax (FP32: two padded vectors of 144)
  T* shift = pub + 3 * kNmax;         // 64
  T* A = shift + 64;                  // n x ld; FP32: reflector rows R overlay it
  T* Zs = A + fast_region_a<T>(n);    // r vectors of length n, padded to n + 1
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const T* L = Lg + (long long)b * sL;

  // L copied row by row with coalesced loads, then symmetrised in place,
  // A = (L + L^T) / 2: the pair {a, c}, a <= c, by one thread (same values as
  // forming each element from L directly; the column reads have pitch n + 1)
  bool bad = false;
  for (int a = warp; a < n; a += kThreads / 32)
    for (int c = lane; c < n; c += 32)
      A[a * ld + c] = guard_ok(gd, L + (long long)a * n + c, sizeof(T), 0x601)
                          ? L[(long long)a * n + c]
                          : T(0);
  __syncthreads();
  for (int a = warp; a < n; a += kThreads / 32)
    for (int c = a + lane; c < n; c += 32) {
      const T x = T(0.5) * (A[a * ld + c] + A[c * ld + a]);
      if (!isfinite(x)) bad = true;
      A[a * ld + c] = x;
      A[c * ld + a] = x;
    }
  if (__syncthreads_or(bad)) {
    for (int idx = tid; idx < n * r; idx += kThreads)
      if (guard_ok(gd, Ug + (long long)b * sU + idx, sizeof(T), 0x602))
        Ug[(long long)b * sU + idx] = T(0);
    if (Utg)
      for (int idx = tid; idx < n * r; idx += kThreads)
        if (guard_ok(gd, Utg + (long long)b * sUt + idx, sizeof(T), 0x603))
          Utg[(long long)b * sUt + idx] = T(0);
    if (tid == 0 && guard_ok(gd, status + b, 4, 0x605)) status[b] = TN_ERR_NONFINITE;
    return;
  }

  // ---- 1. Householder tridiagonalisation
  if constexpr (sizeof(T) == 4) {
    tridiag_regs_f32(reinterpret_cast<float*>(A), ld, n, reinterpret_cast<float*>(A),
                     reinterpret_cast<float*>(dd),
                     reinterpret_cast<float*>(ee), reinterpret_cast<float*>(tau),
                     reinterpret_cast<float*>(vb), reinterpret_cast<float*>(wv),
                     reinterpret_cast<float*>(pub), reinterpret_cast<float*>(part));
  } else {
  const int ri = tid & 127, half = tid >> 7;
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;
    if (warp == 0) {
      T s = T(0);
      for (int j = 1 + lane; j < m; j += 32) {
        const T x = A[(k + 1 + j) * ld + k];
        s += x * x;
      }
      s = warp_sum(s);
      const T alpha = A[(k + 1) * ld + k];
      T tk, beta, sc;
      if (s == T(0)) {
        tk = T(0); beta = alpha; sc = T(0);
      } else {
        beta = -copysign(sqrt(alpha * alpha + s), alpha);
        tk = (beta - alpha) / beta;
        sc = T(1) / (alpha - beta);
      }
      for (int j = lane; j < m; j += 32) {
        const T x = (j == 0) ? T(1) : (tk == T(0) ? T(0) : A[(k + 1 + j) * ld + k] * sc);
        vb[j] = x;
        A[(k + 1 + j) * ld + k] = x;
      }
      if (lane == 0) {
        dd[k] = A[k * ld + k];
        ee[k] = beta;
        tau[k] = tk;
      }
    }
    __syncthreads();
    const T tk = tau[k];
    if (tk == T(0)) continue;  // uniform across the block
    const int c0 = half ? (m + 1) / 2 : 0, c1 = half ? m : (m + 1) / 2;
    if (ri < m) {
      const T* row = A + (k + 1 + ri) * ld + (k + 1);
      T s0 = T(0), s1 = T(0);
      int c = c0;
      for (; c + 1 < c1; c += 2) {
        s0 += row[c] * vb[c];
        s1 += row[c + 1] * vb[c + 1];
      }
      if (c < c1) s0 += row[c] * vb[c];
      part[half * kNmax + ri] = s0 + s1;
    }
    __syncthreads();
    if (warp == 0) {
      T d = T(0);
      for (int i = lane; i < m; i += 32) {
        const T wi = tk * (part[i] + part[kNmax + i]);
        wv[i] = wi;
        d += vb[i] * wi;
      }
      d = warp_sum(d);
      const T K = T(-0.5) * tk * d;
      for (int i = lane; i < m; i += 32) wv[i] += K * vb[i];
    }
    __syncthreads();
    if (ri < m) {
      const T vi = vb[ri], wi = wv[ri];
      T* row = A + (k + 1 + ri) * ld + (k + 1);
      for (int c = c0; c < c1; ++c) row[c] -= vi * wv[c] + wi * vb[c];
    }
    __syncthreads();
  }
  }
  if (tid == 0) {
    if constexpr (sizeof(T) == 8) {  // the FP32 version wrote them from registers
      if (n >= 2) {
        dd[n - 2] = A[(n - 2) * ld + (n - 2)];
        ee[n - 2] = A[(n - 1) * ld + (n - 2)];
        tau[n - 2] = T(0);
      }
      dd[n - 1] = A[(n - 1) * ld + (n - 1)];
      ee[n - 1] = T(0);
    }
    T gl = dd[0], gu = dd[0], emax = T(0);
    for (int j = 0; j < n; ++j) {
      const T el = (j > 0) ? fabs(ee[j - 1]) : T(0);
      const T er = (j + 1 < n) ? fabs(ee[j]) : T(0);
      gl = fmin(gl, dd[j] - el - er);
      gu = fmax(gu, dd[j] + el + er);
      if (j + 1 < n) {
        e2[j] = ee[j] * ee[j];
        emax = fmax(emax, e2[j]);
      }
    }
    const T tnorm = fmax(fabs(gl), fabs(gu));
    const T eps = Lim<T>::eps();
    const T pivmin = Lim<T>::safmin() * fmax(T(1), emax);
    gl -= T(2.1) * tnorm * eps * n + T(4.2) * pivmin;
    gu += T(2.1) * tnorm * eps * n + T(4.2) * pivmin;
    scal[1] = gl;
    scal[2] = gu;
    scal[3] = tnorm;
    scal[4] = pivmin;
  }
  __syncthreads();
  const T gl = scal[1], gu = scal[2], tnorm = scal[3], pivmin = scal[4];
  const T eps = Lim<T>::eps();

  // ---- 2. multisection: 4 threads per eigenvalue
  if constexpr (sizeof(T) == 4) {
    // each thread evaluates kSturmIlp interleaved Sturm sequences, so a round
    // cuts the interval into P + 1 = 4 kSturmIlp + 1 parts; the quad counts
    // the points at or below eigenvalue j (counts are monotone in x) and keeps
    // the part between the last such point and the next
    constexpr int P = 4 * kSturmIlp;
    const int q = tid & 3;
    // a first round shared by all eigenvalues: counts at kThreads equispaced
    // points give each one a starting interval of width (gu - gl) / (kThreads + 1)
    int* gcnt = reinterpret_cast<int*>(part);
    const float hg = (gu - gl) / float(kThreads + 1);
    gcnt[tid] = sturm_count_fast(dd, e2, n, fmaf(hg, float(tid + 1), gl), pivmin);
    __syncthreads();
    for (int base = 0; base < nl; base += kThreads / 4) {
      const int t = base + (tid >> 2);
      const bool valid = (t < nl) && (t < n);
      const int j = n - 1 - t;
      int m0 = 0, m1 = kThreads;  // first grid point whose count exceeds j
      for (int it = 0; it < 9; ++it) {  // 257 outcomes; mid < m1 <= kThreads
        if (m0 >= m1) break;
        const int mid = (m0 + m1) >> 1;
        if (gcnt[mid] <= j) m0 = mid + 1;
        else m1 = mid;
      }
      float lo = (m0 > 0) ? fmaf(hg, float(m0), gl) : gl;
      float hi = (m0 < kThreads) ? fmaf(hg, float(m0 + 1), gl) : gu;
      for (int it = 0; it < kSturmRounds; ++it) {
        const float h = (hi - lo) / float(P + 1);
        float xs[kSturmIlp];
        int cnt[kSturmIlp];
#pragma unroll
        for (int i = 0; i < kSturmIlp; ++i) xs[i] = fmaf(h, float(q + 4 * i + 1), lo);
        if (valid) sturm_count_multi(dd, e2, n, xs, pivmin, cnt);
        int m = 0;
#pragma unroll
        for (int i = 0; i < kSturmIlp; ++i) m += (valid && cnt[i] <= j);
        m += __shfl_xor_sync(0xffffffffu, m, 1);
        m += __shfl_xor_sync(0xffffffffu, m, 2);
        const float nlo = (m > 0) ? fmaf(h, float(m), lo) : lo;
        hi = (m < P) ? fmaf(h, float(m + 1), lo) : hi;
        lo = nlo;
      }
      if (valid && q == 0) lam[t] = 0.5f * (lo + hi);
    }
  } else {
    // interval shrinks 5x per round
    const int q = tid & 3;
    const int rounds = 24;
    for (int base = 0; base < nl; base += kThreads / 4) {
      const int t = base + (tid >> 2);
      const bool valid = (t < nl) && (t < n);
      const int j = n - 1 - t;
      T lo = gl, hi = gu;
      for (int it = 0; it < rounds; ++it) {
        const T h = (hi - lo) / T(5);
        const T x = lo + h * T(q + 1);
        const int cnt = valid ? sturm_count_fast(dd, e2, n, x, pivmin) : 0;
        const int qb = lane & ~3;
        const int n0 = __shfl_sync(0xffffffffu, cnt, qb);
        const int n1 = __shfl_sync(0xffffffffu, cnt, qb + 1);
        const int n2 = __shfl_sync(0xffffffffu, cnt, qb + 2);
        const int n3 = __shfl_sync(0xffffffffu, cnt, qb + 3);
        const T x0 = lo + h, x1 = lo + h * T(2), x2 = lo + h * T(3), x3 = lo + h * T(4);
        if (n0 > j) { hi = x0; }
        else if (n1 > j) { lo = x0; hi = x1; }
        else if (n2 > j) { lo = x1; hi = x2; }
        else if (n3 > j) { lo = x2; hi = x3; }
        else { lo = x3; }
      }
      if (valid && q == 0) lam[t] = T(0.5) * (lo + hi);
    }
  }
  __syncthreads();
  if (tid == 0) {
    const T pertol = T(10) * eps * fmax(tnorm, Lim<T>::safmin());
    for (int t = 0; t < r; ++t) {
      T s = lam[t];
      if (t > 0 && shift[t - 1] - s < pertol) s = shift[t - 1] - pertol;
      shift[t] = s;
    }
  }
  __syncthreads();

  // ---- 3. inverse iteration, one thread per eigenvector: two solves of
  // (T - lambda I) x = y with partial pivoting, the elimination applied to the
  // right-hand side as the factorisation proceeds; the first from a fixed
  // pseudo-random vector, the second from its normalised result, so the
  // contamination by other eigenvectors falls like (eps ||T|| / gap)^2;
  // clusters are separated by the Gram-Schmidt pass below.  y and x live in
  // this thread's padded shared-memory column, the triangular factor (each
  // row divided by its pivot) in local memory.  The pivot choice is made by
  // selects, so the lanes of a warp never diverge.  The solve grows like
  // 1 / (eps ||T||) and L_v carries an arbitrary overall scale, so each
  // solution is brought to max-abs 1 (before Gram-Schmidt squares it) by its
  // reader: the second solve and the vector load take y times vscale.
  const int zld = n + 1;
  T* vscale = shift;  // shift[tid] is read once, before the solves
  if (tid < r) {
    T u2[kNmax], u3[kNmax];
    T* y = Zs + tid * zld;
    auto start = [&](int k) {
      unsigned int h = 2654435761u * (unsigned)(k + 1) ^ (40503u * (unsigned)(tid + 7));
      h ^= h >> 13; h *= 0x5bd1e995u; h ^= h >> 15;
      return T(1) + T(0.5) * (T(h & 0xffff) / T(65536) - T(0.5));
    };
    const T lmb = shift[tid];
    const T tp = fmax(eps * tnorm, Lim<T>::safmin());
    T inv = T(1);  // max-abs normalisation of the previous solve's result
    for (int it = 0; it < 2; ++it) {
    T a = dd[0] - lmb;
    T bb = (n > 1) ? ee[0] : T(0);
    T yk = (it == 0) ? start(0) : y[0] * inv;
    for (int k = 0; k + 1 < n; ++k) {
      const T c = ee[k];
      const T nd = dd[k + 1] - lmb;
      const T ns = (k + 2 < n) ? ee[k + 1] : T(0);
      const T yn = (it == 0) ? start(k + 1) : y[k + 1] * inv;
      // pivot on row k when |a| >= |c| (then a == 0 implies c == 0: use tp)
      const bool piv = fabs(a) >= fabs(c);
      const T den = piv ? ((a == T(0)) ? tp : a) : c;
      const T rd = fdiv(T(1), den);
      const T mlt = (piv ? c : a) * rd;
      const T yo = piv ? yk : yn, ye = piv ? yn : yk;
      u2[k] = (piv ? bb : nd) * rd;
      u3[k] = piv ? T(0) : ns * rd;
      y[k] = yo * rd;
      yk = ye - mlt * yo;
      a = piv ? (nd - mlt * bb) : (bb - mlt * nd);
      bb = piv ? ns : -mlt * ns;
    }
    if (a == T(0)) a = tp;
    T x2 = fdiv(yk, a);  // x_{k+2}, x_{k+1} rolling
    y[n - 1] = x2;
    T x1 = x2;
    T mx = fabs(x2);
    if (n >= 2) {
      x1 = y[n - 2] - u2[n - 2] * x2;
      y[n - 2] = x1;
      mx = fmax(mx, fabs(x1));
    }
#pragma unroll 16
    for (int k = n - 3; k >= 0; --k) {
      const T xk = y[k] - u2[k] * x1 - u3[k] * x2;
      y[k] = xk;
      mx = fmax(mx, fabs(xk));
      x2 = x1;
      x1 = xk;
    }
    inv = (mx > T(0) && isfinite(mx)) ? T(1) / mx : T(1);
    }  // two solves: contamination (eps ||T|| / gap)^2
    vscale[tid] = inv;
  }
  __syncthreads();

  if constexpr (sizeof(T) == 4) {
    vectors_f32(reinterpret_cast<const float*>(Zs), zld,
                reinterpret_cast<const float*>(vscale), n, r,
                reinterpret_cast<const float*>(A), reinterpret_cast<const float*>(tau),
                reinterpret_cast<float*>(pub), reinterpret_cast<float*>(Ug) + (long long)b * sU,
                Utg ? reinterpret_cast<float*>(Utg) + (long long)b * sUt : nullptr, gd);
  } else {
  // ---- 4. vectors into registers: thread = (column c, quarter q of the rows)
  const int col = tid >> 2, qr = tid & 3;
  const bool live = col < r;
  T z[kQ];
#pragma unroll
  for (int kk = 0; kk < kQ; ++kk) {
    const int row = kk * 4 + qr;
    z[kk] = (live && row < n) ? Zs[col * zld + row] * vscale[col] : T(0);
  }
  // modified Gram-Schmidt in descending eigenvalue order
  for (int j = 0; j < r; ++j) {
    if (col == j) {
      T s = T(0);
#pragma unroll
      for (int kk = 0; kk < kQ; ++kk) s += z[kk] * z[kk];
      s = quad_sum(s);
      const T inv = (s > T(0)) ? T(1) / sqrt(s) : T(0);
#pragma unroll
      for (int kk = 0; kk < kQ; ++kk) {
        z[kk] *= inv;
        pub[kk * 4 + qr] = z[kk];
      }
    }
    __syncthreads();
    if (live && col > j) {
      T d = T(0);
#pragma unroll
      for (int kk = 0; kk < kQ; ++kk) d += pub[kk * 4 + qr] * z[kk];
      d = quad_sum(d);
#pragma unroll
      for (int kk = 0; kk < kQ; ++kk) z[kk] -= d * pub[kk * 4 + qr];
    }
    __syncthreads();
  }
  // back-transformation by the stored reflectors (v_k in column k below the diagonal)
  for (int k = n - 3; k >= 0; --k) {
    const T tk = tau[k];
    if (tk == T(0)) continue;
    T vk[kQ];
    T d = T(0);
#pragma unroll
    for (int kk = 0; kk < kQ; ++kk) {
      const int row = kk * 4 + qr;
      vk[kk] = (row > k && row < n) ? A[row * ld + k] : T(0);
      d += vk[kk] * z[kk];
    }
    d = quad_sum(d) * tk;
#pragma unroll
    for (int kk = 0; kk < kQ; ++kk) z[kk] -= d * vk[kk];
  }
  // sign: largest-|.| entry (first on ties) positive
  {
    T best = T(-1);
    int bi = kNmax;
#pragma unroll
    for (int kk = 0; kk < kQ; ++kk) {
      const int row = kk * 4 + qr;
      const T a = fabs(z[kk]);
      if (row < n && (a > best || (a == best && row < bi))) { best = a; bi = row; }
    }
    const unsigned qm = 0xFu << (threadIdx.x & 28);
    for (int o = 1; o <= 2; o <<= 1) {
      const T ob = __shfl_xor_sync(qm, best, o);
      const int oi = __shfl_xor_sync(qm, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    // the owner of row bi tells the quad its sign
    T sv = T(0);
#pragma unroll
    for (int kk = 0; kk < kQ; ++kk)
      if (kk * 4 + qr == bi) sv = z[kk];
    sv = quad_sum(sv);
    const T sgn = (sv < T(0)) ? T(-1) : T(1);
#pragma unroll
    for (int kk = 0; kk < kQ; ++kk) z[kk] *= sgn;
  }
  if (live) {
    T* U = Ug + (long long)b * sU;
#pragma unroll
    for (int kk = 0; kk < kQ; ++kk) {
      const int row = kk * 4 + qr;
      if (row < n) U[(long long)row * r + col] = z[kk];
    }
    if (Utg) {
      T* Ut = Utg + (long long)b * sUt + (long long)col * n;
#pragma unroll
      for (int kk = 0; kk < kQ; ++kk) {
        const int row = kk * 4 + qr;
        if (row < n) Ut[row] = z[kk];
      }
    }
  }
  }
  if (lamg) {
    double* lo = lamg + (long long)b * slam;
    for (int t = tid; t < nlam && t < n; t += kThreads)
      if (guard_ok(gd, lo + t, 8, 0x609)) lo[t] = double(lam[t]);
  }
}

template <typename T>
size_t eigh_fast_smem_bytes(int n, int r) {
  // dd ee e2 tau vb wv (6), part (2), lam (1), pub (3), shift (64), then A, Z
  return sizeof(T) * (size_t(fast_region_a<T>(n)) + size_t(r) * (n + 1) + 12 * kNmax + 64);
}

}  // namespace

template <typename T>
size_t eigh_smem_bytes(int n, int r, int nlam) {
  const int nl = nlam > r ? nlam : r;
  return sizeof(T) * (size_t(n) * (n + 1) + size_t(n) * r + 7 * size_t(n) + nl + r);
}

template <typename T>
cudaError_t launch_eigh_top(const T* L, long long sL, T* U, long long sU, T* Ut, long long sUt,
                            double* lam, long long slam, int n, int r, int nlam, int* status,
                            int batch, cudaStream_t st) {
  if (n < 1 || n > kNmax || r < 1 || r > n || nlam > n) return cudaErrorInvalidValue;
  const size_t fast_smem = eigh_fast_smem_bytes<T>(n, r);
  if (r <= 64 && fast_smem <= eigh_fast_smem_limit<T>()) {
    k_eigh_fast<T><<<batch, kThreads, fast_smem, st>>>(L, sL, U, sU, Ut, sUt, lam, slam, n, r,
                                                       nlam, status, nullptr);
    return cudaGetLastError();
  }
  const size_t smem = eigh_smem_bytes<T>(n, r, nlam);
  if (smem > eigh_smem_limit<T>()) return cudaErrorInvalidValue;
  k_eigh_top<T, T><<<batch, kThreads, smem, st>>>(L, sL, U, sU, Ut, sUt, lam, slam, n, r, nlam,
                                                  status);
  return cudaGetLastError();
}

namespace {
size_t g_limit[5] = {0, 0, 0, 0, 0};  // top<double>, top<float>, fast<double>, fast<float>,
                                      // fast<float> grouped

template <typename K>
cudaError_t configure_kernel(K kern, size_t* out) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa{};
  e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return e;
  const size_t lim = size_t(optin) - fa.sharedSizeBytes;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(lim));
  if (e == cudaSuccess) *out = lim;
  return e;
}
}  // namespace

template <typename T>
size_t eigh_smem_limit() {
  return g_limit[sizeof(T) == 8 ? 0 : 1];
}
template <typename T>
size_t eigh_fast_smem_limit() {
  return g_limit[sizeof(T) == 8 ? 2 : 3];
}
template size_t eigh_smem_limit<double>();
template size_t eigh_smem_limit<float>();
template size_t eigh_fast_smem_limit<double>();
template size_t eigh_fast_smem_limit<float>();

cudaError_t eigh_configure() {
  cudaError_t e = configure_kernel(k_eigh_top<double, double>, &g_limit[0]);
  if (e == cudaSuccess) e = configure_kernel(k_eigh_top<float, float>, &g_limit[1]);
  if (e == cudaSuccess) e = configure_kernel(k_eigh_fast<double>, &g_limit[2]);
  if (e == cudaSuccess) e = configure_kernel(k_eigh_fast<float>, &g_limit[3]);
  size_t lim1 = 0, lim2 = 0;
  if (e == cudaSuccess) e = configure_kernel(k_eigh_fast<float, 1>, &lim1);
  if (e == cudaSuccess) e = configure_kernel(k_eigh_fast<float, 2>, &lim2);
  if (e == cudaSuccess) g_limit[4] = std::min(lim1, lim2);
  return e;
}

cudaError_t launch_eigh_grouped(const EighDesc* desc, int n_prob, int max_n, int max_r,
                                bool guarded, cudaStream_t st) {
  if (n_prob <= 0) return cudaSuccess;
  if (max_n < 1 || max_n > kNmax || max_r < 1 || max_r > 64) return cudaErrorInvalidValue;
  const size_t smem = eigh_fast_smem_bytes<float>(max_n, max_r);
  if (smem > g_limit[4]) return cudaErrorInvalidValue;
  auto kern = guarded ? k_eigh_fast<float, 2> : k_eigh_fast<float, 1>;
  kern<<<n_prob, kThreads, smem, st>>>(nullptr, 0, nullptr, 0, nullptr, 0, nullptr, 0, 0, 0, 0,
                                       nullptr, desc);
  return cudaGetLastError();
}

template size_t eigh_smem_bytes<double>(int, int, int);
template size_t eigh_smem_bytes<float>(int, int, int);
template cudaError_t launch_eigh_top<double>(const double*, long long, double*, long long, double*,
                                             long long, double*, long long, int, int, int, int*,
                                             int, cudaStream_t);
template cudaError_t launch_eigh_top<float>(const float*, long long, float*, long long, float*,
                                            long long, double*, long long, int, int, int, int*,
                                            int, cudaStream_t);

}  // namespace tn
