// FP64 kernels of the density-matrix tree approximation: site normalisation,
// block fusion, batched contractions, root renormalisation and the closing
// contraction of the last partition.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "kernels.cuh"
#include "tn_dmtree.h"

namespace tn {

namespace {

__device__ __forceinline__ double block_sum(double v, double* red) {
  // Fixed-order tree reduction over a 256-thread block (deterministic).
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) red[0] = t;
  }
  __syncthreads();
  return red[0];
}

__device__ __forceinline__ double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_down_sync(0xffffffffu, t, o));
    if (threadIdx.x == 0) red[0] = t;
  }
  __syncthreads();
  return red[0];
}

// ---------------------------------------------------------------- site norms
// Every site tensor is scaled to unit Frobenius norm; ln of the norms is summed
// into the instance's FP64 log-scale in a fixed order.
__global__ void __launch_bounds__(256) k_site_norm(const double* const* tens, const int64_t* off,
                                                   const int64_t* len, int nv, double* inv_norm,
                                                   double* logscale, int* status) {
  __shared__ double red[32];
  const int i = blockIdx.x;
  const double* T = tens[i];
  double lsum = 0.0;
  bool bad = false;
  for (int v = threadIdx.x; v < nv; v += blockDim.x) {
    const double* t = T + off[v];
    double ss = 0.0;
    for (int64_t j = 0; j < len[v]; ++j) ss = fma(t[j], t[j], ss);
    const double nrm = sqrt(ss);
    if (!(nrm > 0.0) || !isfinite(nrm)) bad = true;
    inv_norm[(long long)i * nv + v] = (nrm > 0.0) ? 1.0 / nrm : 0.0;
    lsum += log(nrm);
  }
  const double tot = block_sum(lsum, red);
  const int anybad = __syncthreads_or(bad);
  if (threadIdx.x == 0) {
    logscale[i] = tot;
    status[i] = anybad ? TN_ERR_NONFINITE : TN_OK;
  }
}

// ---------------------------------------------------------------- fusion
__global__ void __launch_bounds__(256) k_fuse(const FuseSite* __restrict__ sites,
                                              const double* const* tens,
                                              const double* __restrict__ inv_norm, int nv,
                                              const double* __restrict__ S, long long sS,
                                              int trivial, double* __restrict__ Y, long long sY) {
  const FuseSite f = sites[blockIdx.y];
  const int i = blockIdx.z;
  const long long total = (long long)f.a * f.dhl * f.de * f.b * f.dhr;
  const long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= total) return;
  // o -> (a, hl, e, b, hr), row-major
  long long t = o;
  const int hr = int(t % f.dhr); t /= f.dhr;
  const int bb = int(t % f.b);   t /= f.b;
  const int e = int(t % f.de);   t /= f.de;
  const int hl = int(t % f.dhl); t /= f.dhl;
  const int aa = int(t);
  const double* T = tens[i] + f.t_off + hl * f.shl + hr * f.shr + e * f.se;
  double acc = 0.0;
  if (trivial) {
    acc = T[0];
  } else {
    const double* Sk = S + (long long)i * sS + f.s_off + (long long)aa * f.dp * f.b + bb;
    for (int p = 0; p < f.dp; ++p) acc = fma(Sk[(long long)p * f.b], T[p * f.sp], acc);
  }
  Y[(long long)i * sY + f.y_off + o] = acc * inv_norm[(long long)i * nv + f.vertex];
}

// ---------------------------------------------------------------- DGEMM
constexpr int BM = 64, BN = 64, BK = 16;

template <bool TA, bool TB>
__global__ void __launch_bounds__(256) k_dgemm(GemmArgs g) {
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const int i = blockIdx.z;
  const double* A = g.A + (long long)i * g.sA;
  const double* B = g.B + (long long)i * g.sB;
  double* C = g.C + (long long)i * g.sC;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  for (int k0 = 0; k0 < g.K; k0 += BK) {
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int idx = tid + 256 * l;
      int mm, kk;
      if (!TA) { mm = idx >> 4; kk = idx & 15; } else { mm = idx & 63; kk = idx >> 6; }
      const int gm = m0 + mm, gk = k0 + kk;
      double v = 0.0;
      if (gm < g.M && gk < g.K) v = TA ? A[(long long)gk * g.lda + gm] : A[(long long)gm * g.lda + gk];
      As[kk][mm] = v;
      int nn;
      if (!TB) { nn = idx & 63; kk = idx >> 6; } else { kk = idx & 15; nn = idx >> 4; }
      const int gn = n0 + nn;
      const int gk2 = k0 + kk;
      double w = 0.0;
      if (gn < g.N && gk2 < g.K) w = TB ? B[(long long)gn * g.ldb + gk2] : B[(long long)gk2 * g.ldb + gn];
      Bs[kk][nn] = w;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) { a[q] = As[kk][ty + 16 * q]; b[q] = Bs[kk][tx + 16 * q]; }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fma(a[p], b[q], acc[p][q]);
    }
    __syncthreads();
  }
  double alpha = 1.0;
  if (g.amax_in) {
    const double mx = __longlong_as_double((long long)g.amax_in[(long long)i * g.s_amax_in]);
    alpha = (mx > 0.0) ? 1.0 / mx : 1.0;
  }
  double lmax = 0.0;
  bool nan_seen = false;
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int gm = m0 + ty + 16 * p;
    if (gm >= g.M) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int gn = n0 + tx + 16 * q;
      if (gn >= g.N) continue;
      const double v = alpha * acc[p][q];
      C[(long long)gm * g.ldc + gn] = v;
      lmax = fmax(lmax, fabs(v));
      nan_seen |= isnan(v);
    }
  }
  if (g.amax_out) {
    if (nan_seen) lmax = INFINITY;
    for (int o = 16; o > 0; o >>= 1) lmax = fmax(lmax, __shfl_down_sync(0xffffffffu, lmax, o));
    if ((tid & 31) == 0) {
      unsigned long long bits = (unsigned long long)__double_as_longlong(lmax);
      atomicMax(g.amax_out + (long long)i * g.s_amax_out, bits);
    }
  }
}

// ---------------------------------------------------------------- env root
__global__ void k_fill_env_root(double* R, long long sR, unsigned long long* amax, long long s_amax,
                                int batch) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= batch) return;
  R[(long long)i * sR] = 1.0;
  amax[(long long)i * s_amax] = (unsigned long long)__double_as_longlong(1.0);
}

// ---------------------------------------------------------------- root
// M_r = P (r x D) . Y (D x d); unit Frobenius norm; log-scale += ln ||M_r||.
// Also writes the identity boundary site of the first leg (1, d0, d0).
__global__ void __launch_bounds__(256) k_root(const double* P, long long sP, const double* Y,
                                              long long sY, int r, int D, int d, double* S_root,
                                              double* S_first, int d0, long long sS,
                                              double* logscale, int* status) {
  __shared__ double red[32];
  extern __shared__ double mr[];
  const int i = blockIdx.x;
  const double* Pi = P + (long long)i * sP;
  const double* Yi = Y + (long long)i * sY;
  double ss = 0.0;
  for (int o = threadIdx.x; o < r * d; o += blockDim.x) {
    const int a = o / d, e = o % d;
    double acc = 0.0;
    for (int k = 0; k < D; ++k) acc = fma(Pi[(long long)a * D + k], Yi[(long long)k * d + e], acc);
    mr[o] = acc;
    ss = fma(acc, acc, ss);
  }
  const double tot = block_sum(ss, red);
  const double nrm = sqrt(tot);
  const double inv = (nrm > 0.0) ? 1.0 / nrm : 0.0;
  double* Si = S_root + (long long)i * sS;
  for (int o = threadIdx.x; o < r * d; o += blockDim.x) Si[o] = mr[o] * inv;
  double* Fi = S_first + (long long)i * sS;
  for (int o = threadIdx.x; o < d0 * d0; o += blockDim.x) Fi[o] = (o / d0 == o % d0) ? 1.0 : 0.0;
  if (threadIdx.x == 0) {
    if (!(nrm > 0.0) || !isfinite(nrm)) {
      if (status[i] == TN_OK) status[i] = TN_ERR_NONFINITE;
    } else {
      logscale[i] += log(nrm);
    }
  }
}

// ---------------------------------------------------------------- closing
// The last contraction has no open legs: s = Y_0 Y_1 ... Y_{n-1} (vectors
// times D x D matrices), renormalised at every site; ln Z = ln s + log-scale.
__global__ void __launch_bounds__(256) k_close(const double* Y, long long sY, const int64_t* y_off,
                                               const int32_t* D, int n, const double* logscale,
                                               double* logz, int* status) {
  __shared__ double red[32];
  extern __shared__ double vbuf[];
  const int i = blockIdx.x;
  const double* Yi = Y + (long long)i * sY;
  int Dl = D[0];
  double* v = vbuf;
  double* w = vbuf + D[n];  // D[n] holds maxD
  for (int o = threadIdx.x; o < Dl; o += blockDim.x) v[o] = Yi[y_off[0] + o];
  __syncthreads();
  double lsum = 0.0;
  for (int k = 1; k < n; ++k) {
    const int Dr = D[k];
    const double* Yk = Yi + y_off[k];
    double lm = 0.0;
    for (int c = threadIdx.x; c < Dr; c += blockDim.x) {
      double acc = 0.0;
      for (int a = 0; a < Dl; ++a) acc = fma(v[a], Yk[(long long)a * Dr + c], acc);
      w[c] = acc;
      lm = fmax(lm, fabs(acc));
    }
    const double mx = block_max(lm, red);
    const double inv = (mx > 0.0) ? 1.0 / mx : 1.0;
    if (mx > 0.0) lsum += log(mx);
    for (int c = threadIdx.x; c < Dr; c += blockDim.x) v[c] = w[c] * inv;
    __syncthreads();
    Dl = Dr;
  }
  if (threadIdx.x == 0) {
    const double s = v[0];
    int st = status[i];
    if (st == TN_OK && !isfinite(s)) st = TN_ERR_NONFINITE;
    if (st == TN_OK && !(s > 0.0)) st = TN_ERR_NONPOSITIVE;
    status[i] = st;
    logz[i] = (st == TN_OK) ? log(s) + lsum + logscale[i] : NAN;
  }
}

}  // namespace

cudaError_t launch_dgemm(bool ta, bool tb, const GemmArgs& g, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return cudaSuccess;
  dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, g.batch);
  if (!ta && !tb) k_dgemm<false, false><<<grid, 256, 0, st>>>(g);
  else if (!ta && tb) k_dgemm<false, true><<<grid, 256, 0, st>>>(g);
  else if (ta && !tb) k_dgemm<true, false><<<grid, 256, 0, st>>>(g);
  else k_dgemm<true, true><<<grid, 256, 0, st>>>(g);
  return cudaGetLastError();
}

cudaError_t launch_site_norm(const double* const* tens, const int64_t* off, const int64_t* len,
                             int nv, int batch, double* inv_norm, double* logscale, int* status,
                             cudaStream_t st) {
  k_site_norm<<<batch, 256, 0, st>>>(tens, off, len, nv, inv_norm, logscale, status);
  return cudaGetLastError();
}

cudaError_t launch_fuse(const FuseSite* sites, int n, int max_elems, const double* const* tens,
                        const double* inv_norm, int nv, const double* S, long long sS,
                        int trivial, double* Y, long long sY, int batch, cudaStream_t st) {
  dim3 grid((max_elems + 255) / 256, n, batch);
  k_fuse<<<grid, 256, 0, st>>>(sites, tens, inv_norm, nv, S, sS, trivial, Y, sY);
  return cudaGetLastError();
}

cudaError_t launch_fill_env_root(double* R, long long sR, unsigned long long* amax,
                                 long long s_amax, int batch, cudaStream_t st) {
  k_fill_env_root<<<(batch + 127) / 128, 128, 0, st>>>(R, sR, amax, s_amax, batch);
  return cudaGetLastError();
}

cudaError_t launch_root(const double* P, long long sP, const double* Y, long long sY, int r, int D,
                        int d, double* S_root, double* S_first, int d0, long long sS,
                        double* logscale, int* status, int batch, cudaStream_t st) {
  const size_t smem = sizeof(double) * size_t(r) * d;
  k_root<<<batch, 256, smem, st>>>(P, sP, Y, sY, r, D, d, S_root, S_first, d0, sS, logscale,
                                   status);
  return cudaGetLastError();
}

cudaError_t launch_close(const double* Y, long long sY, const int64_t* y_off, const int32_t* D,
                         int n, int maxD, const double* logscale, double* logz, int* status,
                         int batch, cudaStream_t st) {
  const size_t smem = sizeof(double) * size_t(2 * maxD);
  if (smem > 48 * 1024) {  // wide closing chains of general plans (maxD <= 4096)
    const cudaError_t e =
        cudaFuncSetAttribute(k_close, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
  }
  k_close<<<batch, 256, smem, st>>>(Y, sY, y_off, D, n, logscale, logz, status);
  return cudaGetLastError();
}

}  // namespace tn
