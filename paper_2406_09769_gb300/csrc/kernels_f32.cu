// FP32-storage kernels of the mixed-precision path: block fusion (also writing
// the transposed block used as a K-major tensor-core operand), the root tensor
// with its FP64 norm, and the closing contraction.  Sums that feed ln Z are
// accumulated in FP64.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "kernels.cuh"
#include "tn_dmtree.h"

namespace tn {

namespace {

__device__ __forceinline__ double block_sum_d(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) red[0] = t;
  }
  __syncthreads();
  return red[0];
}

__device__ __forceinline__ double block_max_d(double v, double* red) {
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

// Y[a, hl, e, b, hr] = inv_norm * sum_p S[a, p, b] T[p, hl, hr, e]  (FP32 arithmetic: a
// sum over the bond dimension p, rounded once to the FP32 storage precision; FP64 units
// are a small fraction of FP32 ones on this part) and, when Yt is set,
// Yt[(e * Dr + b * dhr + hr) * Dl + a * dhl + hl] = same value.
__global__ void __launch_bounds__(256) k_fuse_f32(const FuseSite* __restrict__ sites,
                                                  const double* const* tens,
                                                  const double* __restrict__ inv_norm, int nv,
                                                  const float* __restrict__ S, long long sS,
                                                  int trivial, float* __restrict__ Y, long long sY,
                                                  float* __restrict__ Yt, const int64_t* yt_off) {
  const FuseSite f = sites[blockIdx.y];
  const int i = blockIdx.z;
  const long long total = (long long)f.a * f.dhl * f.de * f.b * f.dhr;
  const long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= total) return;
  long long t = o;
  const int hr = int(t % f.dhr); t /= f.dhr;
  const int bb = int(t % f.b);   t /= f.b;
  const int e = int(t % f.de);   t /= f.de;
  const int hl = int(t % f.dhl); t /= f.dhl;
  const int aa = int(t);
  const double* T = tens[i] + f.t_off + hl * f.shl + hr * f.shr + e * f.se;
  float acc = 0.f;
  if (trivial) {
    acc = float(T[0]);
  } else {
    const float* Sk = S + (long long)i * sS + f.s_off + (long long)aa * f.dp * f.b + bb;
    for (int p = 0; p < f.dp; ++p) acc = fmaf(Sk[(long long)p * f.b], float(T[p * f.sp]), acc);
  }
  const float v = acc * float(inv_norm[(long long)i * nv + f.vertex]);
  Y[(long long)i * sY + f.y_off + o] = v;
  if (Yt) {
    const long long Dl = (long long)f.a * f.dhl, Dr = (long long)f.b * f.dhr;
    const long long row = (long long)e * Dr + (long long)bb * f.dhr + hr;
    Yt[(long long)i * sY + yt_off[blockIdx.y] + row * Dl + (long long)aa * f.dhl + hl] = v;
  }
}

// Same fusion, tiled for the transposed copy: block (32 x 8) owns a 32 x 32 tile
// of Ymat[a'][j] (a' = a * dhl + hl, j = e * Dr + b * dhr + hr); Y is written
// along j and Yt along a', both coalesced, through a shared-memory tile.
// grid: (ceil(d*Dr / 32), ceil(Dl / 32), sites * batch), z = instance * sites + site.
__global__ void __launch_bounds__(256) k_fuse_f32_tiled(const FuseSite* __restrict__ sites,
                                                        int n_sites, const double* const* tens,
                                                        const double* __restrict__ inv_norm,
                                                        int nv, const float* __restrict__ S,
                                                        long long sS, float* __restrict__ Y,
                                                        long long sY, float* __restrict__ Yt,
                                                        const int64_t* yt_off) {
  __shared__ float tile[32][33];
  const int site = blockIdx.z % n_sites, i = blockIdx.z / n_sites;
  const FuseSite f = sites[site];
  const int Dl = f.a * f.dhl, Dr = f.b * f.dhr, J = f.de * Dr;
  const int j0 = blockIdx.x * 32, a0 = blockIdx.y * 32;
  if (j0 >= J || a0 >= Dl) return;  // uniform per block
  const double* Tb = tens[i] + f.t_off;
  const float* Si = S + (long long)i * sS + f.s_off;
  const float inv = float(inv_norm[(long long)i * nv + f.vertex]);
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int j = j0 + tx;
  int e = 0, bb = 0, hr = 0;
  if (j < J) {
    e = j / Dr;
    const int c = j - e * Dr;
    bb = c / f.dhr;
    hr = c - bb * f.dhr;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int ap = a0 + ty + 8 * q;
    float v = 0.f;
    if (j < J && ap < Dl) {
      const int aa = ap / f.dhl, hl = ap - aa * f.dhl;
      const double* T = Tb + hl * f.shl + hr * f.shr + e * f.se;
      const float* Sk = Si + (long long)aa * f.dp * f.b + bb;
      float acc = 0.f;
      for (int p = 0; p < f.dp; ++p) acc = fmaf(Sk[(long long)p * f.b], float(T[p * f.sp]), acc);
      v = acc * inv;
      Y[(long long)i * sY + f.y_off + (long long)ap * J + j] = v;
    }
    tile[ty + 8 * q][tx] = v;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int jj = j0 + ty + 8 * q, ap = a0 + tx;
    if (jj < J && ap < Dl)
      Yt[(long long)i * sY + yt_off[site] + (long long)jj * Dl + ap] = tile[tx][ty + 8 * q];
  }
}

// Wider tile of the same fusion: block of 256 threads owns 32 rows a' x 128
// columns j; thread (c, g) = (tid % 32, tid / 32) computes j = j0 + c + 32 u and
// a' = a0 + g + 8 q (u, q = 0..3), so every Y store instruction writes 32
// consecutive j of one row, and Yt is written from a [32][129] shared tile
// (odd stride: conflict-free column reads) along a'.  The site tensor's
// (at most kFuseT) entries are staged as FP32 in shared memory.
constexpr int kFuseT = 256;
__global__ void __launch_bounds__(256) k_fuse_f32_wide(const FuseSite* __restrict__ sites,
                                                       int n_sites, const double* const* tens,
                                                       const double* __restrict__ inv_norm,
                                                       int nv, const float* __restrict__ S,
                                                       long long sS, float* __restrict__ Y,
                                                       long long sY, float* __restrict__ Yt,
                                                       const int64_t* yt_off) {
  __shared__ float tile[32][129];
  __shared__ float ts[kFuseT];
  const int site = blockIdx.z % n_sites, i = blockIdx.z / n_sites;
  const FuseSite f = sites[site];
  const int Dl = f.a * f.dhl, Dr = f.b * f.dhr, J = f.de * Dr;
  const int j0 = blockIdx.x * 128, a0 = blockIdx.y * 32;
  if (j0 >= J || a0 >= Dl) return;  // uniform per block
  const int tid = threadIdx.x, c = tid & 31, g = tid >> 5;
  // T[p][hl][hr][e] (strides sp, shl, shr, se) staged densely as [p][hl][hr][e]
  const int nT = f.dp * f.dhl * f.dhr * f.de;
  const double* Tb = tens[i] + f.t_off;
  for (int q = tid; q < nT; q += 256) {
    int t = q;
    const int e = t % f.de; t /= f.de;
    const int hr = t % f.dhr; t /= f.dhr;
    const int hl = t % f.dhl; t /= f.dhl;
    ts[q] = float(Tb[t * f.sp + hl * f.shl + hr * f.shr + e * f.se]);
  }
  __syncthreads();
  const float* Si = S + (long long)i * sS + f.s_off;
  const float inv = float(inv_norm[(long long)i * nv + f.vertex]);
  const int tp = f.dhl * f.dhr * f.de;  // stride of p in ts
  int jb[4], jt[4];                     // per column: S offset (b), ts offset (hr, e)
  bool jok[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int j = j0 + c + 32 * u;
    jok[u] = j < J;
    const int e = jok[u] ? j / Dr : 0;
    const int cc = jok[u] ? j - e * Dr : 0;
    const int bb = cc / f.dhr, hr = cc - bb * f.dhr;
    jb[u] = bb;
    jt[u] = hr * f.de + e;
  }
  float* Yi = Y + (long long)i * sY + f.y_off;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int ap = a0 + g + 8 * q;
    const bool aok = ap < Dl;
    const int aa = aok ? ap / f.dhl : 0, hl = aok ? ap - aa * f.dhl : 0;
    const float* Sk = Si + (long long)aa * f.dp * f.b;
    const int tb = hl * f.dhr * f.de;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      float v = 0.f;
      if (aok && jok[u]) {
        float acc = 0.f;
        for (int p = 0; p < f.dp; ++p)
          acc = fmaf(Sk[(long long)p * f.b + jb[u]], ts[p * tp + tb + jt[u]], acc);
        v = acc * inv;
        Yi[(long long)ap * J + j0 + c + 32 * u] = v;
      }
      tile[g + 8 * q][c + 32 * u] = v;
    }
  }
  if (!Yt) return;  // uniform
  __syncthreads();
  float* Yti = Yt + (long long)i * sY + yt_off[site];
  const int ap = a0 + c;
  for (int jj = g; jj < 128; jj += 8) {
    const int j = j0 + jj;
    if (j < J && ap < Dl) Yti[(long long)j * Dl + ap] = tile[c][jj];
  }
}

// The same fusion when every bond of the site is of dimension 2 (dp = dhl =
// dhr = de = 2: Dl = 2a, Dr = 2b, J = 4b), as on the square lattices.  Block
// of 256 threads owns a = aa0 .. aa0 + 15 and b = bb0 .. bb0 + 63; thread (x,
// y) = (tid % 64, tid / 64) reads S[aa, 0, bb] and S[aa, 1, bb] for bb = bb0 +
// x and aa = aa0 + y + 4 m (m = 0..3) and forms the 2 x 2 x 2 block
// Y[2 aa + hl][e * 2b + 2 bb + hr] from the 16 site-tensor entries held in
// registers: each S value feeds eight outputs, and the hr pairs are float2
// stores (consecutive threads write consecutive pairs of one row).  Yt is
// written from a shared tile [32 rows a'][2 x 128 columns j] (pitch 258:
// float2-aligned rows) along a', 32 consecutive a' per warp store.  A site
// with other bond dimensions or an odd Y offset (the end sites of a row have
// dhl = 1 or dhr = 1) takes a plain per-element path over the same (a, b)
// range.  grid: (ceil(max b / 64), ceil(max a / 16), sites * batch).
constexpr int kFuseD2Pitch = 258;
__global__ void __launch_bounds__(256) k_fuse_f32_d2(const FuseSite* __restrict__ sites,
                                                     int n_sites, const double* const* tens,
                                                     const double* __restrict__ inv_norm, int nv,
                                                     const float* __restrict__ S, long long sS,
                                                     float* __restrict__ Y, long long sY,
                                                     float* __restrict__ Yt,
                                                     const int64_t* yt_off) {
  __shared__ __align__(16) float tile[32 * kFuseD2Pitch];
  const int site = blockIdx.z % n_sites, i = blockIdx.z / n_sites;
  const FuseSite f = sites[site];
  const int bb0 = blockIdx.x * 64, aa0 = blockIdx.y * 16;
  if (bb0 >= f.b || aa0 >= f.a) return;  // uniform per block
  const int tid = threadIdx.x, x = tid & 63, y = tid >> 6;
  const double* Tb = tens[i] + f.t_off;
  const float inv = float(inv_norm[(long long)i * nv + f.vertex]);
  const float* Si = S + (long long)i * sS + f.s_off;
  float* Yi = Y + (long long)i * sY + f.y_off;
  float* Yti = Yt + (long long)i * sY + yt_off[site];
  if (f.dp != 2 || f.dhl != 2 || f.dhr != 2 || f.de != 2 || (f.y_off & 1) || (yt_off[site] & 1)) {
    const int Dl = f.a * f.dhl, Dr = f.b * f.dhr, J = f.de * Dr;
    const int per = f.dhl * f.dhr * f.de;
    for (int q = tid; q < 16 * 64 * per; q += 256) {
      int r = q;
      const int e = r % f.de; r /= f.de;
      const int hr = r % f.dhr; r /= f.dhr;
      const int hl = r % f.dhl; r /= f.dhl;
      const int bb = bb0 + r % 64, aa = aa0 + r / 64;
      if (aa >= f.a || bb >= f.b) continue;
      const double* T = Tb + hl * f.shl + hr * f.shr + e * f.se;
      const float* Sk = Si + (long long)aa * f.dp * f.b + bb;
      float acc = 0.f;
      for (int p = 0; p < f.dp; ++p) acc = fmaf(Sk[(long long)p * f.b], float(T[p * f.sp]), acc);
      const float v = acc * inv;
      const int ap = aa * f.dhl + hl, j = e * Dr + bb * f.dhr + hr;
      Yi[(long long)ap * J + j] = v;
      Yti[(long long)j * Dl + ap] = v;
    }
    return;  // uniform per block
  }
  const int Dl = 2 * f.a, J = 4 * f.b;
  float t[2][2][2][2];  // [p][hl][hr][e]
#pragma unroll
  for (int p = 0; p < 2; ++p)
#pragma unroll
    for (int hl = 0; hl < 2; ++hl)
#pragma unroll
      for (int hr = 0; hr < 2; ++hr)
#pragma unroll
        for (int e = 0; e < 2; ++e)
          t[p][hl][hr][e] = float(Tb[p * f.sp + hl * f.shl + hr * f.shr + e * f.se]);
  const int bb = bb0 + x;
  const bool bok = bb < f.b;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const int al = y + 4 * m, aa = aa0 + al;
    const bool ok = bok && aa < f.a;
    const float s0 = ok ? Si[(long long)aa * 2 * f.b + bb] : 0.f;
    const float s1 = ok ? Si[(long long)aa * 2 * f.b + f.b + bb] : 0.f;
#pragma unroll
    for (int hl = 0; hl < 2; ++hl)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        // sum over p in the order of the other fusion kernels, then the site norm
        const float v0 = fmaf(s1, t[1][hl][0][e], s0 * t[0][hl][0][e]) * inv;
        const float v1 = fmaf(s1, t[1][hl][1][e], s0 * t[0][hl][1][e]) * inv;
        const float2 v = make_float2(v0, v1);
        if (ok)
          *reinterpret_cast<float2*>(Yi + (long long)(2 * aa + hl) * J + e * 2 * f.b + 2 * bb) = v;
        *reinterpret_cast<float2*>(tile + (2 * al + hl) * kFuseD2Pitch + e * 128 + 2 * x) = v;
      }
  }
  __syncthreads();
  // Yt[j][a'] for the block's 2 x 128 columns j and 32 rows a'
  const int lane = tid & 31, w = tid >> 5, ap = 2 * aa0 + lane;
  for (int jl = w; jl < 256; jl += 8) {
    const int e = jl >> 7, c = jl & 127;  // column 2 bb0 + c of half e
    if (2 * bb0 + c < 2 * f.b && ap < Dl)
      Yti[(long long)(e * 2 * f.b + 2 * bb0 + c) * Dl + ap] = tile[lane * kFuseD2Pitch + jl];
  }
}

__global__ void k_fill_env_root_f32(float* R, long long sR, unsigned int* amax, long long s_amax,
                                    int batch) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= batch) return;
  R[(long long)i * sR] = 1.0f;
  amax[(long long)i * s_amax] = __float_as_uint(1.0f);
}

// M_r = P (r x D) . Y (D x d), FP64 accumulation and norm; unit-norm FP32
// store; log-scale += ln ||M_r||; identity boundary site of the first leg.
// kMode 0: strided batch; 1: grouped (block i runs problem desc[i]); 2: as 1
// with the range guard checked on every global access.
template <int kMode>
__global__ void __launch_bounds__(256) k_root_f32(const float* P_, long long sP, int ldp_,
                                                  const float* Y_, long long sY, int r_, int D_,
                                                  int d_, float* S_root_, float* S_first_, int d0_,
                                                  long long sS, double* logscale_, int* status_,
                                                  const RootDesc* __restrict__ desc) {
  __shared__ double red[32];
  extern __shared__ double mr[];
  // grouped launch: block i runs problem desc[i] with its own pointers and
  // shape; else instance blockIdx.x of the strided arguments
  const RootDesc* q = kMode ? desc + blockIdx.x : nullptr;
  const GuardTab* gd = kMode == 2 ? q->guard : nullptr;
  const int i = q ? 0 : int(blockIdx.x);
  const float* Pi = q ? q->P : P_ + (long long)i * sP;
  const float* Yi = q ? q->Y : Y_ + (long long)i * sY;
  float* Si = q ? q->S_root : S_root_ + (long long)i * sS;
  float* Fi = q ? q->S_first : S_first_ + (long long)i * sS;
  double* logscale = q ? q->logscale : logscale_;
  int* status = q ? q->status : status_;
  const int ldp = q ? q->ldp : ldp_, r = q ? q->r : r_, D = q ? q->D : D_, d = q ? q->d : d_;
  const int d0 = q ? q->d0 : d0_;
  double ss = 0.0;
  for (int o = threadIdx.x; o < r * d; o += blockDim.x) {
    const int a = o / d, e = o % d;
    double acc = 0.0;
    for (int k = 0; k < D; ++k) {
      const float* pp = Pi + (long long)a * ldp + k;
      const float* py = Yi + (long long)k * d + e;
      if (guard_ok(gd, pp, 4, 0x701) && guard_ok(gd, py, 4, 0x702))
        acc = fma((double)*pp, (double)*py, acc);
    }
    mr[o] = acc;
    ss = fma(acc, acc, ss);
  }
  const double nrm = sqrt(block_sum_d(ss, red));
  const double inv = (nrm > 0.0) ? 1.0 / nrm : 0.0;
  for (int o = threadIdx.x; o < r * d; o += blockDim.x)
    if (guard_ok(gd, Si + o, 4, 0x703)) Si[o] = float(mr[o] * inv);
  for (int o = threadIdx.x; o < d0 * d0; o += blockDim.x)
    if (guard_ok(gd, Fi + o, 4, 0x704)) Fi[o] = (o / d0 == o % d0) ? 1.f : 0.f;
  if (threadIdx.x == 0 && guard_ok(gd, status + i, 4, 0x705) &&
      guard_ok(gd, logscale + i, 8, 0x706)) {
    if (!(nrm > 0.0) || !isfinite(nrm)) {
      if (status[i] == TN_OK) status[i] = TN_ERR_NONFINITE;
    } else {
      logscale[i] += log(nrm);
    }
  }
}

__global__ void __launch_bounds__(256) k_close_f32(const float* Y, long long sY, const int64_t* y_off,
                                                   const int32_t* D, int n, const double* logscale,
                                                   double* logz, int* status) {
  __shared__ double red[32];
  extern __shared__ double vbuf[];
  const int i = blockIdx.x;
  const float* Yi = Y + (long long)i * sY;
  int Dl = D[0];
  double* v = vbuf;
  double* w = vbuf + D[n];
  for (int o = threadIdx.x; o < Dl; o += blockDim.x) v[o] = Yi[y_off[0] + o];
  __syncthreads();
  double lsum = 0.0;
  for (int k = 1; k < n; ++k) {
    const int Dr = D[k];
    const float* Yk = Yi + y_off[k];
    double lm = 0.0;
    for (int c = threadIdx.x; c < Dr; c += blockDim.x) {
      double acc = 0.0;
      for (int a = 0; a < Dl; ++a) acc = fma(v[a], (double)Yk[(long long)a * Dr + c], acc);
      w[c] = acc;
      lm = fmax(lm, fabs(acc));
    }
    const double mx = block_max_d(lm, red);
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

// C_i = alpha_i * A_i B_i^T for shapes the TMA path cannot address (leading
// dimensions that are not a multiple of 16 bytes); one thread per output,
// FP64 accumulation.  Same argument semantics as the tensor-core kernel.
__global__ void __launch_bounds__(256) k_sgemm_nt(TcGemmArgs g) {
  const int i = blockIdx.z;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = idx < (long long)g.M * g.N;
  float x = 0.f;
  if (live) {
    const int m = int(idx / g.N), n = int(idx % g.N);
    const float* a = g.A + (long long)i * g.sA + (long long)m * g.lda;
    const float* b = g.B + (long long)i * g.sB + (long long)n * g.ldb;
    double acc = 0.0;
    for (int k = 0; k < g.K; ++k) acc = fma((double)a[k], (double)b[k], acc);
    float alpha = 1.f;
    if (g.amax_in) {
      const float mx = __uint_as_float(g.amax_in[(long long)i * g.s_amax_in]);
      alpha = (mx > 0.f) ? 1.f / mx : 1.f;
    }
    x = float(acc) * alpha;
    if (g.C) g.C[(long long)i * g.sC + (long long)m * g.ldc + n] = x;
    if (g.Ct) {
      const int q = n / g.ct_cols, cc = n - q * g.ct_cols;
      g.Ct[(long long)i * g.sCt + (long long)cc * g.ldct + (long long)m * (g.N / g.ct_cols) + q] = x;
    }
  }
  if (g.amax_out) {
    float v = live ? (isfinite(x) ? fabsf(x) : INFINITY) : 0.f;
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) atomicMax(g.amax_out + (long long)i * g.s_amax_out, __float_as_uint(v));
  }
}

// C_i = alpha_i A_i B_i^T in FP32 with FFMA accumulation (round to nearest
// at every step, so the rounding errors have no common sign), for the value
// path of the mixed precision: on this part the tcgen05 FP32 accumulator
// drops low bits (a relative bias of about -1e-8 per accumulated MMA, growing
// with K), and a bias of one sign in the tree tensors compounds over the
// vertices of a pass and over passes into ln Z.  64 x 64 tile per block of
// 256 threads (4 x 4 per thread), K in chunks of 16 staged transposed in
// shared memory.
// kComp: compensated (Kahan) accumulation, y = fma(a, b, -c) rounded once
// per term and the running sum's rounding carried in c: the dot product is
// then accurate to a few eps of sqrt(sum of squared terms), like an FP64
// accumulation of the FP32 products, at four FP32 operations per term.
constexpr int kSgT = 64, kSgK = 16;
// kMode 0: batch of strided problems (blockIdx.z = instance of g_in);
// 1: grouped launch, blockIdx.z = problem desc[z] with its own pointers and
// shape (tiles beyond a problem's extent return at once); 2: as 1 with the
// range guard of the descriptors checked on every global access.
template <bool kComp, int kMode>
__global__ void __launch_bounds__(256) k_sgemm_ffma(TcGemmArgs g_in,
                                                    const GemmDesc* __restrict__ desc) {
  __shared__ float As[kSgK][kSgT + 4];
  __shared__ float Bs[kSgK][kSgT + 4];
  __shared__ float red[8];
  // the problem's operands: its descriptor (grouped launch, blockIdx.z =
  // problem) or batch entry blockIdx.z of the strided arguments
  const int z = blockIdx.z;
  const GemmDesc* dz = kMode ? desc + z : nullptr;
  const GuardTab* gd = kMode == 2 ? dz->guard : nullptr;
  const int M = dz ? dz->M : g_in.M;
  const int N = dz ? dz->N : g_in.N;
  const int K = dz ? dz->K : g_in.K;
  const int lda = dz ? dz->lda : g_in.lda;
  const int ldb = dz ? dz->ldb : g_in.ldb;
  const int ldc = dz ? dz->ldc : g_in.ldc;
  const int ldct = dz ? dz->ldct : g_in.ldct;
  const int ct_cols = dz ? dz->ct_cols : g_in.ct_cols;
  const float* A = dz ? dz->A : g_in.A + (long long)z * g_in.sA;
  const float* B = dz ? dz->B : g_in.B + (long long)z * g_in.sB;
  float* C = dz ? dz->C : (g_in.C ? g_in.C + (long long)z * g_in.sC : nullptr);
  float* Ct = dz ? dz->Ct : (g_in.Ct ? g_in.Ct + (long long)z * g_in.sCt : nullptr);
  const unsigned int* amax_in =
      dz ? dz->amax_in : (g_in.amax_in ? g_in.amax_in + (long long)z * g_in.s_amax_in : nullptr);
  unsigned int* amax_out =
      dz ? dz->amax_out
         : (g_in.amax_out ? g_in.amax_out + (long long)z * g_in.s_amax_out : nullptr);
  const int m0 = blockIdx.y * kSgT, n0 = blockIdx.x * kSgT;
  if (m0 >= M || n0 >= N) return;  // uniform per block
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const bool vec = (lda % 4 == 0) && (ldb % 4 == 0) &&
                   (reinterpret_cast<uintptr_t>(A) % 16 == 0) &&
                   (reinterpret_cast<uintptr_t>(B) % 16 == 0);
  const int lr = tid >> 2, lk = (tid & 3) * 4;  // loader: row, first k of its 4
  float acc[4][4], cmp[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = cmp[u][v] = 0.f;
  for (int k0 = 0; k0 < K; k0 += kSgK) {
    float av[4], bv[4];
    const int am = m0 + lr, bn = n0 + lr, kk = k0 + lk;
    if (vec && kk + 3 < K) {
      const float* pa = A + (long long)am * lda + kk;
      const float* pb = B + (long long)bn * ldb + kk;
      const float4 a4 = (am < M && guard_ok(gd, pa, 16, 0x201))
                            ? *reinterpret_cast<const float4*>(pa)
                            : make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 b4 = (bn < N && guard_ok(gd, pb, 16, 0x202))
                            ? *reinterpret_cast<const float4*>(pb)
                            : make_float4(0.f, 0.f, 0.f, 0.f);
      av[0] = a4.x; av[1] = a4.y; av[2] = a4.z; av[3] = a4.w;
      bv[0] = b4.x; bv[1] = b4.y; bv[2] = b4.z; bv[3] = b4.w;
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float* pa = A + (long long)am * lda + kk + q;
        const float* pb = B + (long long)bn * ldb + kk + q;
        av[q] = (am < M && kk + q < K && guard_ok(gd, pa, 4, 0x203)) ? *pa : 0.f;
        bv[q] = (bn < N && kk + q < K && guard_ok(gd, pb, 4, 0x204)) ? *pb : 0.f;
      }
    }
    __syncthreads();  // the previous chunk's reads are done
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      As[lk + q][lr] = av[q];
      Bs[lk + q][lr] = bv[q];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kSgK; ++k) {
      const float4 a = *reinterpret_cast<const float4*>(&As[k][4 * ty]);
      const float4 b = *reinterpret_cast<const float4*>(&Bs[k][4 * tx]);
      const float ar[4] = {a.x, a.y, a.z, a.w}, br[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          if (kComp) {
            const float y = fmaf(ar[u], br[v], -cmp[u][v]);
            const float t = acc[u][v] + y;
            cmp[u][v] = (t - acc[u][v]) - y;
            acc[u][v] = t;
          } else {
            acc[u][v] = fmaf(ar[u], br[v], acc[u][v]);
          }
        }
    }
  }
  float alpha = 1.f;
  if (amax_in && guard_ok(gd, amax_in, 4, 0x207)) {
    const float mx = __uint_as_float(*amax_in);
    alpha = (mx > 0.f) ? 1.f / mx : 1.f;
  }
  float lmax = 0.f;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int m = m0 + 4 * ty + u;
    if (m >= M) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int n = n0 + 4 * tx + v;
      if (n >= N) continue;
      const float x = acc[u][v] * alpha;
      float* pc = C ? C + (long long)m * ldc + n : nullptr;
      if (pc && guard_ok(gd, pc, 4, 0x205)) *pc = x;
      if (Ct) {
        const int q = n / ct_cols, cc = n - q * ct_cols;
        float* pt = Ct + (long long)cc * ldct + (long long)m * (N / ct_cols) + q;
        if (guard_ok(gd, pt, 4, 0x206)) *pt = x;
      }
      lmax = fmaxf(lmax, isfinite(x) ? fabsf(x) : INFINITY);
    }
  }
  if (amax_out) {
    for (int o = 16; o > 0; o >>= 1) lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
    if ((tid & 31) == 0) red[tid >> 5] = lmax;
    __syncthreads();
    if (tid == 0) {
      float v = red[0];
      for (int w = 1; w < 8; ++w) v = fmaxf(v, red[w]);
      if (guard_ok(gd, amax_out, 4, 0x208)) atomicMax(amax_out, __float_as_uint(v));
    }
  }
}

}  // namespace

cudaError_t launch_sgemm_nt(const TcGemmArgs& g, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return cudaSuccess;
  if (g.Ct && (g.ct_cols <= 0 || g.N % g.ct_cols)) return cudaErrorInvalidValue;
  const long long tot = (long long)g.M * g.N;
  dim3 grid(unsigned((tot + 255) / 256), 1, g.batch);
  k_sgemm_nt<<<grid, 256, 0, st>>>(g);
  return cudaGetLastError();
}

cudaError_t launch_sgemm_ffma(const TcGemmArgs& g, bool compensated, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return cudaSuccess;
  if (g.Ct && (g.ct_cols <= 0 || g.N % g.ct_cols)) return cudaErrorInvalidValue;
  dim3 grid(unsigned((g.N + kSgT - 1) / kSgT), unsigned((g.M + kSgT - 1) / kSgT), g.batch);
  if (compensated) k_sgemm_ffma<true, 0><<<grid, 256, 0, st>>>(g, nullptr);
  else k_sgemm_ffma<false, 0><<<grid, 256, 0, st>>>(g, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_gemm_grouped(const GemmDesc* desc, int n_prob, int max_M, int max_N,
                                bool compensated, bool guarded, cudaStream_t st) {
  if (n_prob <= 0 || max_M <= 0 || max_N <= 0) return cudaSuccess;
  if (n_prob > 65535) return cudaErrorInvalidValue;
  TcGemmArgs g{};
  dim3 grid(unsigned((max_N + kSgT - 1) / kSgT), unsigned((max_M + kSgT - 1) / kSgT),
            unsigned(n_prob));
  if (guarded) {
    if (compensated) k_sgemm_ffma<true, 2><<<grid, 256, 0, st>>>(g, desc);
    else k_sgemm_ffma<false, 2><<<grid, 256, 0, st>>>(g, desc);
  } else {
    if (compensated) k_sgemm_ffma<true, 1><<<grid, 256, 0, st>>>(g, desc);
    else k_sgemm_ffma<false, 1><<<grid, 256, 0, st>>>(g, desc);
  }
  return cudaGetLastError();
}

cudaError_t launch_fuse_f32(const FuseSite* sites, int n, int max_elems, int max_dl, int max_j,
                            int max_t, int max_a, int max_b, int bond2,
                            const double* const* tens,
                            const double* inv_norm, int nv, const float* S, long long sS,
                            int trivial, float* Y, long long sY, float* Yt, const int64_t* yt_off,
                            int batch, cudaStream_t st) {
  if (Yt && !trivial && max_dl > 0 && max_j > 0) {
    if (bond2 && sY % 2 == 0 && max_a > 0 && max_b > 0) {
      dim3 grid((max_b + 63) / 64, (max_a + 15) / 16, n * batch);
      k_fuse_f32_d2<<<grid, 256, 0, st>>>(sites, n, tens, inv_norm, nv, S, sS, Y, sY, Yt, yt_off);
      return cudaGetLastError();
    }
    if (max_t <= kFuseT) {
      dim3 grid((max_j + 127) / 128, (max_dl + 31) / 32, n * batch);
      k_fuse_f32_wide<<<grid, 256, 0, st>>>(sites, n, tens, inv_norm, nv, S, sS, Y, sY, Yt,
                                            yt_off);
      return cudaGetLastError();
    }
    dim3 grid((max_j + 31) / 32, (max_dl + 31) / 32, n * batch);
    k_fuse_f32_tiled<<<grid, dim3(32, 8), 0, st>>>(sites, n, tens, inv_norm, nv, S, sS, Y, sY, Yt,
                                                   yt_off);
    return cudaGetLastError();
  }
  dim3 grid((max_elems + 255) / 256, n, batch);
  k_fuse_f32<<<grid, 256, 0, st>>>(sites, tens, inv_norm, nv, S, sS, trivial, Y, sY, Yt, yt_off);
  return cudaGetLastError();
}

cudaError_t launch_fill_env_root_f32(float* R, long long sR, unsigned int* amax, long long s_amax,
                                     int batch, cudaStream_t st) {
  k_fill_env_root_f32<<<(batch + 127) / 128, 128, 0, st>>>(R, sR, amax, s_amax, batch);
  return cudaGetLastError();
}

cudaError_t launch_root_f32(const float* P, long long sP, int ldp, const float* Y, long long sY,
                            int r, int D, int d, float* S_root, float* S_first, int d0,
                            long long sS, double* logscale, int* status, int batch,
                            cudaStream_t st) {
  const size_t smem = sizeof(double) * size_t(r) * d;
  k_root_f32<0><<<batch, 256, smem, st>>>(P, sP, ldp, Y, sY, r, D, d, S_root, S_first, d0, sS,
                                       logscale, status, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_root_grouped(const RootDesc* desc, int n_prob, int max_rd, bool guarded,
                                cudaStream_t st) {
  if (n_prob <= 0) return cudaSuccess;
  const size_t smem = sizeof(double) * size_t(max_rd);
  if (smem > 48 * 1024) return cudaErrorInvalidValue;
  auto kern = guarded ? k_root_f32<2> : k_root_f32<1>;
  kern<<<n_prob, 256, smem, st>>>(nullptr, 0, 0, nullptr, 0, 0, 0, 0, nullptr, nullptr, 0,
                                        0, nullptr, nullptr, desc);
  return cudaGetLastError();
}

namespace {
__global__ void k_env_root_grouped(const EnvRootDesc* __restrict__ desc, int n_prob) {
  const int p = blockIdx.x;
  if (p >= n_prob) return;
  const EnvRootDesc q = desc[p];
  for (int k = threadIdx.x; k < q.n; k += blockDim.x)
    if (guard_ok(q.guard, q.amax + k, 4, 0x101))
      q.amax[k] = (k == q.n - 1) ? __float_as_uint(1.0f) : 0u;
  if (threadIdx.x == 0 && guard_ok(q.guard, q.R, 4, 0x102)) q.R[0] = 1.0f;
}
}  // namespace

cudaError_t launch_env_root_grouped(const EnvRootDesc* desc, int n_prob, cudaStream_t st) {
  if (n_prob <= 0) return cudaSuccess;
  k_env_root_grouped<<<n_prob, 64, 0, st>>>(desc, n_prob);
  return cudaGetLastError();
}

cudaError_t launch_close_f32(const float* Y, long long sY, const int64_t* y_off, const int32_t* D,
                             int n, int maxD, const double* logscale, double* logz, int* status,
                             int batch, cudaStream_t st) {
  const size_t smem = sizeof(double) * size_t(2 * maxD);
  if (smem > 48 * 1024) {  // wide closing chains of general plans (maxD <= 4096)
    const cudaError_t e =
        cudaFuncSetAttribute(k_close_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
  }
  k_close_f32<<<batch, 256, smem, st>>>(Y, sY, y_off, D, n, logscale, logz, status);
  return cudaGetLastError();
}

namespace {
// One segment per tree position: a rows x cols row-major matrix at src_off of
// every instance's source buffer, converted to dst_off of its destination
// buffer (and, with dst_t, its transpose at the same offset of dst_t).
template <typename S, typename D>
__global__ void __launch_bounds__(256) k_convert_segments(const S* const* src_tab,
                                                          const S* src_base, long long s_src,
                                                          D* const* dst_tab, D* dst_base,
                                                          long long s_dst, D* dst_t,
                                                          const CvtSeg* __restrict__ segs) {
  const CvtSeg sg = segs[blockIdx.y];
  const int i = blockIdx.z;
  const S* src = (src_tab ? src_tab[i] : src_base + (long long)i * s_src) + sg.src_off;
  D* dst = (dst_tab ? dst_tab[i] : dst_base + (long long)i * s_dst) + sg.dst_off;
  D* dt = dst_t ? dst_t + (long long)i * s_dst + sg.dst_off : nullptr;
  const long long total = (long long)sg.rows * sg.cols;
  for (long long idx = blockIdx.x * 256ll + threadIdx.x; idx < total;
       idx += 256ll * gridDim.x) {
    const D x = D(src[idx]);
    dst[idx] = x;
    if (dt) {
      const long long r = idx / sg.cols, c = idx - r * sg.cols;
      dt[c * sg.rows + r] = x;
    }
  }
}
}  // namespace

cudaError_t launch_convert_segments_d2f(const double* const* src_tab, float* dst_base,
                                        long long s_dst, float* dst_t, const CvtSeg* segs,
                                        int nseg, int max_elems, int batch, cudaStream_t st) {
  if (nseg < 1 || batch < 1) return cudaSuccess;
  dim3 grid((max_elems + 255) / 256, nseg, batch);
  k_convert_segments<double, float><<<grid, 256, 0, st>>>(src_tab, nullptr, 0, nullptr, dst_base,
                                                          s_dst, dst_t, segs);
  return cudaGetLastError();
}

cudaError_t launch_convert_segments_f2d(const float* src_base, long long s_src,
                                        double* const* dst_tab, const CvtSeg* segs, int nseg,
                                        int max_elems, int batch, cudaStream_t st) {
  if (nseg < 1 || batch < 1) return cudaSuccess;
  dim3 grid((max_elems + 255) / 256, nseg, batch);
  k_convert_segments<float, double><<<grid, 256, 0, st>>>(nullptr, src_base, s_src, dst_tab,
                                                          nullptr, 0, nullptr, segs);
  return cudaGetLastError();
}

}  // namespace tn
