// Learned per-edge rank allocation (no counterpart in the paper).
//
// After the eigensolver of tree vertex v, a small MLP maps spectrum features of
// L_v to a rank chi_v <= r_v (the structural rank of the chi_max plan) under a
// per-pass budget sum_v chi_v <= sum_v min(chi_u, r_v) (the total rank of the
// uniform-chi_u method).  Columns of U_v beyond chi_v are zeroed, so shapes stay
// those of the chi_max plan and the tree TN has rank chi_v on that edge.
//
// dim A is the effective one, chi_{v-1} d_v (the rows of M_v that the ranks
// kept so far can fill); the plan's rows beyond it are zero.
// Features of one edge (22): log10(lam_k / lam_1) / 30 at k = 2, 4, 8, 12, 16,
// 24, 32, 48, 64, 96, 128 (clamped to dim A), log10 of the discarded share
// sum_{i >= r} lam_i / sum lam at r = 8, 16, 24, 32, 48, 64 (divided by 30),
// both floored at 1e-12 (below the eigensolver's resolution), dim A / 128,
// v / (n - 1), pass / passes, the pass budget still unspent per edge left
// (this one included) / 64, and the uniform method's rank min(chi_u, r_v) / 64.
// MLP: 22 -> 64 -> 64 -> 1 with ReLU; BF16 weights, FP32 accumulation;
// chi = clamp(rint(64 y), 1, min(r_v, numerical rank)), the numerical rank
// being the last index with lam_i > 1e-12 lam_1, then lowered so that each
// later vertex u of the pass keeps min(2, r_u) ranks of the budget (rank 1
// would cut all correlations across that edge).  Training: mean squared error against
// offline water-filling labels chi / 64, FP32 master weights, Adam.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "kernels.cuh"

namespace tn {

namespace {

constexpr int F = kRankFeatures;
constexpr int H = kRankHidden;

__device__ __forceinline__ float bfv(const __nv_bfloat16* w, int i) { return __bfloat162float(w[i]); }

// parameter offsets in the flat vector [W1 (H x F), b1, W2 (H x H), b2, W3 (H), b3]
constexpr int oW1 = 0, ob1 = H * F, oW2 = ob1 + H, ob2 = oW2 + H * H, oW3 = ob2 + H, ob3 = oW3 + H;

constexpr double kFloor = 1e-12;

__device__ void edge_features(const double* lam, int A, int v, int nlegs, int pass, int npass,
                              int remaining, int edges_left, int uniform_rank, float* f) {
  const double top = lam[0] > 0.0 ? lam[0] : 1.0;
  double total = 0.0;
  for (int i = 0; i < A; ++i) total += fmax(lam[i], 0.0);
  if (!(total > 0.0)) total = 1.0;
  const int ks[11] = {2, 4, 8, 12, 16, 24, 32, 48, 64, 96, 128};
  for (int q = 0; q < 11; ++q) {
    const int idx = (ks[q] < A ? ks[q] : A) - 1;
    f[q] = float(log10(fmax(fmax(lam[idx], 0.0) / top, kFloor)) / 30.0);
  }
  const int rs[6] = {8, 16, 24, 32, 48, 64};
  for (int q = 0; q < 6; ++q) {
    double d = 0.0;
    if (rs[q] < A) {
      for (int i = rs[q]; i < A; ++i) d += fmax(lam[i], 0.0);
      d /= total;
    }
    f[11 + q] = float(log10(fmax(d, kFloor)) / 30.0);
  }
  f[17] = float(A / 128.0);
  f[18] = float(double(v) / double(nlegs > 1 ? nlegs - 1 : 1));
  f[19] = float(double(pass) / double(npass > 0 ? npass : 1));
  f[20] = float(double(remaining) / double(edges_left) / 64.0);
  f[21] = float(double(uniform_rank) / 64.0);
}

__device__ double disc_share(const double* lam, int A, int chi) {
  double tot = 0.0, d = 0.0;
  for (int i = 0; i < A; ++i) {
    const double x = fmax(lam[i], 0.0);
    tot += x;
    if (i >= chi) d += x;
  }
  return tot > 0.0 ? d / tot : 0.0;
}

// one block (64 threads) per instance
template <typename T>
__global__ void __launch_bounds__(64) k_rank_select(RankArgs g, T* U, long long sU, T* Ut,
                                                    long long sUt) {
  __shared__ float f[F];
  __shared__ float h1[H];
  __shared__ float h2[H];
  __shared__ float ysum[2];
  __shared__ int chi_s;
  const int i = blockIdx.x, t = threadIdx.x;
  const double* lam = g.lam + (long long)i * g.slam;
  // effective dim A_v and structural rank under the ranks kept so far
  const int A = g.first ? g.A : min(g.A, g.prev_chi[i] * g.dk);
  const int rk = min(g.rk, A);
  const int rem0 = g.first ? g.budget_total : g.budget_rem[i];
  if (t == 0)
    edge_features(lam, A, g.v, g.nlegs, g.pass, g.npass, rem0, g.edges_after + 1,
                  min(g.chi_uniform, g.rk), f);
  __syncthreads();
  int chi = rk;
  if (!g.model && g.fixed_chi > 0) chi = min(rk, g.fixed_chi);  // uniform chi (the judge's run)
  if (g.model) {
    const __nv_bfloat16* W = static_cast<const __nv_bfloat16*>(g.model);
    float z = bfv(W, ob1 + t);
    for (int j = 0; j < F; ++j) z = fmaf(bfv(W, oW1 + t * F + j), f[j], z);
    h1[t] = fmaxf(z, 0.f);
    __syncthreads();
    z = bfv(W, ob2 + t);
    for (int j = 0; j < H; ++j) z = fmaf(bfv(W, oW2 + t * H + j), h1[j], z);
    h2[t] = fmaxf(z, 0.f);
    float y = bfv(W, oW3 + t) * h2[t];
    for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
    if ((t & 31) == 0) ysum[t >> 5] = y;
    __syncthreads();
    if (t == 0) {
      const float yy = ysum[0] + ysum[1] + bfv(W, ob3);
      float pred = rintf(64.f * yy);
      if (!(pred >= 1.f)) pred = 1.f;            // also catches NaN
      // never spend budget on eigenvalues below the resolution floor
      int nrank = 1;
      for (int q = 1; q < A; ++q)
        if (lam[q] > kFloor * lam[0]) nrank = q + 1;
      int c = pred > float(rk) ? rk : int(pred);
      if (c > nrank) c = nrank;
      const int allowed = rem0 - g.reserve_after;
      if (c > allowed) c = allowed;
      if (c < 1) c = 1;
      chi_s = c;
    }
    __syncthreads();
    chi = chi_s;
  }
  if (t == 0) {
    g.prev_chi[i] = chi;
    g.budget_rem[i] = rem0 - chi;
    if (g.acc) g.acc[i] += disc_share(lam, A, chi);
    if (g.rec_chi) g.rec_chi[g.rec_off + i] = chi;
    if (g.rec_feat)
      for (int j = 0; j < F; ++j) g.rec_feat[(g.rec_off + i) * F + j] = f[j];
    if (g.rec_spec)
      for (int j = 0; j < 128; ++j) g.rec_spec[(g.rec_off + i) * 128 + j] = j < A ? lam[j] : 0.0;
  }
  if (chi < g.rk) {
    T* Ui = U + (long long)i * sU;
    for (int idx = t; idx < g.A * g.rk; idx += blockDim.x)
      if (idx % g.rk >= chi) Ui[idx] = T(0);
    if (Ut) {
      T* Uti = Ut + (long long)i * sUt;
      for (int idx = t; idx < g.A * g.rk; idx += blockDim.x)
        if (idx / g.A >= chi) Uti[idx] = T(0);
    }
  }
}

// Forward + backward of the MSE over samples [s0, s0 + n) of X (n_total x F),
// S samples per block; the block's gradient is added to grad atomically.
// (16 samples keep the block's static shared memory near 36 KB.)
constexpr int kS = 16;

__global__ void __launch_bounds__(256) k_mlp_grad(const float* __restrict__ X,
                                                  const float* __restrict__ tgt,
                                                  const int* __restrict__ idx, int n, float scale,
                                                  const float* __restrict__ w,
                                                  float* __restrict__ grad, float* __restrict__ loss) {
  __shared__ float Wr[H * H + H * F + 3 * H + 1];  // BF16-rounded weights (forward)
  __shared__ float xs[kS][F];
  __shared__ float z1[kS][H], z2[kS][H];
  __shared__ float dy[kS];
  __shared__ float d2[kS][H];
  const int tid = threadIdx.x;
  const int np = H * F + H + H * H + H + H + 1;
  for (int q = tid; q < np; q += blockDim.x) Wr[q] = __bfloat162float(__float2bfloat16_rn(w[q]));
  const int s0 = blockIdx.x * kS;
  for (int q = tid; q < kS * F; q += blockDim.x) {
    const int s = q / F, j = q % F;
    xs[s][j] = (s0 + s < n) ? X[(long long)idx[s0 + s] * F + j] : 0.f;
  }
  __syncthreads();
  for (int q = tid; q < kS * H; q += blockDim.x) {
    const int s = q / H, u = q % H;
    float z = Wr[ob1 + u];
    for (int j = 0; j < F; ++j) z = fmaf(Wr[oW1 + u * F + j], xs[s][j], z);
    z1[s][u] = z;
  }
  __syncthreads();
  for (int q = tid; q < kS * H; q += blockDim.x) {
    const int s = q / H, u = q % H;
    float z = Wr[ob2 + u];
    for (int j = 0; j < H; ++j) z = fmaf(Wr[oW2 + u * H + j], fmaxf(z1[s][j], 0.f), z);
    z2[s][u] = z;
  }
  __syncthreads();
  if (tid < kS) {
    const int s = tid;
    float y = Wr[ob3];
    for (int u = 0; u < H; ++u) y = fmaf(Wr[oW3 + u], fmaxf(z2[s][u], 0.f), y);
    const bool live = s0 + s < n;
    const float r = live ? y - tgt[idx[s0 + s]] : 0.f;
    dy[s] = 2.f * r * scale;
    atomicAdd(loss, r * r * scale);
  }
  __syncthreads();
  // layer 3
  for (int u = tid; u < H; u += blockDim.x) {
    float g3 = 0.f;
    for (int s = 0; s < kS; ++s) g3 += dy[s] * fmaxf(z2[s][u], 0.f);
    atomicAdd(&grad[oW3 + u], g3);
  }
  if (tid == 0) {
    float gb = 0.f;
    for (int s = 0; s < kS; ++s) gb += dy[s];
    atomicAdd(&grad[ob3], gb);
  }
  for (int q = tid; q < kS * H; q += blockDim.x) {
    const int s = q / H, u = q % H;
    d2[s][u] = (z2[s][u] > 0.f) ? dy[s] * Wr[oW3 + u] : 0.f;
  }
  __syncthreads();
  // layer 2: dW2[u][j] = sum_s d2[s][u] relu(z1[s][j]); db2[u] = sum_s d2[s][u]
  for (int q = tid; q < H * H; q += blockDim.x) {
    const int u = q / H, j = q % H;
    float g2 = 0.f;
    for (int s = 0; s < kS; ++s) g2 += d2[s][u] * fmaxf(z1[s][j], 0.f);
    atomicAdd(&grad[oW2 + q], g2);
  }
  for (int u = tid; u < H; u += blockDim.x) {
    float gb = 0.f;
    for (int s = 0; s < kS; ++s) gb += d2[s][u];
    atomicAdd(&grad[ob2 + u], gb);
  }
  __syncthreads();
  // d1[s][j] = (z1 > 0) * sum_u d2[s][u] W2[u][j]; reuse z2 as d1 storage
  for (int q = tid; q < kS * H; q += blockDim.x) {
    const int s = q / H, j = q % H;
    float a = 0.f;
    for (int u = 0; u < H; ++u) a = fmaf(d2[s][u], Wr[oW2 + u * H + j], a);
    z2[s][j] = (z1[s][j] > 0.f) ? a : 0.f;
  }
  __syncthreads();
  for (int q = tid; q < H * F; q += blockDim.x) {
    const int u = q / F, j = q % F;
    float g1 = 0.f;
    for (int s = 0; s < kS; ++s) g1 += z2[s][u] * xs[s][j];
    atomicAdd(&grad[oW1 + q], g1);
  }
  for (int u = tid; u < H; u += blockDim.x) {
    float gb = 0.f;
    for (int s = 0; s < kS; ++s) gb += z2[s][u];
    atomicAdd(&grad[ob1 + u], gb);
  }
}

// Offline labels: greedy water-filling of one DM pass's rank budget over its
// edges, one warp per (pass, instance).  Starting from chi_e = 1, each step
// gives one more rank to the edge whose next eigenvalue carries the largest
// share of its spectrum (ties: lowest edge); this minimises the summed
// discarded share because each edge's discarded share is convex in chi_e.
// The pass budget is sum_e min(chi_u, cap[e]).  When feat is set, features 20
// and 21 of each edge are rewritten for the labelled allocation (budget left
// before the edge per edge left, uniform rank).
// spec: [(e * B + i) * 128 + j]; edges of pass p are [pass_start[p], pass_start[p + 1]).
constexpr int kWfLane = 8;  // edges per lane: up to 256 edges per pass

__global__ void __launch_bounds__(32) k_water_fill(const double* __restrict__ spec,
                                                   const int* __restrict__ cap,
                                                   const int* __restrict__ pass_start,
                                                   int chi_u, int B, int* __restrict__ chi_out,
                                                   float* __restrict__ feat) {
  const int p = blockIdx.y, i = blockIdx.x, lane = threadIdx.x;
  const int e0 = pass_start[p], ne = pass_start[p + 1] - e0;
  int budget = 0;
  for (int e = lane; e < ne; e += 32) budget += min(chi_u, cap[e0 + e]);
  for (int o = 16; o > 0; o >>= 1) budget += __shfl_xor_sync(0xffffffffu, budget, o);
  int alloc[kWfLane];
  double tot[kWfLane];
#pragma unroll
  for (int q = 0; q < kWfLane; ++q) {
    alloc[q] = 1;
    tot[q] = 0.0;
    const int e = lane + 32 * q;
    if (e < ne) {
      const double* s = spec + ((long long)(e0 + e) * B + i) * 128;
      double t = 0.0;
      for (int j = 0; j < 128; ++j) t += fmax(s[j], 0.0);
      tot[q] = t;
    }
  }
  for (int used = ne; used < budget; ++used) {
    double best = -1.0;
    int be = 0x7fffffff;
#pragma unroll
    for (int q = 0; q < kWfLane; ++q) {
      const int e = lane + 32 * q;
      if (e < ne && alloc[q] < cap[e0 + e] && alloc[q] < 128) {
        const double x = fmax(spec[((long long)(e0 + e) * B + i) * 128 + alloc[q]], 0.0);
        const double gain = tot[q] > 0.0 ? x / tot[q] : 0.0;
        if (gain > best) {
          best = gain;
          be = e;
        }
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oe = __shfl_xor_sync(0xffffffffu, be, o);
      if (ob > best || (ob == best && oe < be)) {
        best = ob;
        be = oe;
      }
    }
    if (be == 0x7fffffff) break;
    if ((be & 31) == lane) {
#pragma unroll
      for (int q = 0; q < kWfLane; ++q)
        if (lane + 32 * q == be) ++alloc[q];
    }
  }
#pragma unroll
  for (int q = 0; q < kWfLane; ++q) {
    const int e = lane + 32 * q;
    if (e < ne) chi_out[(long long)(e0 + e) * B + i] = alloc[q];
  }
  __syncwarp();
  if (feat && lane == 0) {
    int rem = budget;
    for (int j = 0; j < ne; ++j) {
      const long long r = (long long)(e0 + j) * B + i;
      feat[r * kRankFeatures + 20] = float(double(rem) / double(ne - j) / 64.0);
      feat[r * kRankFeatures + 21] = float(double(min(chi_u, cap[e0 + j])) / 64.0);
      rem -= chi_out[r];
    }
  }
}

__global__ void k_iota(int* x, int n) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) x[q] = q;
}

__global__ void k_adam(float* w, float* grad, float* m, float* v, int np, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= np) return;
  const float g = grad[q];
  const float mq = b1 * m[q] + (1.f - b1) * g;
  const float vq = b2 * v[q] + (1.f - b2) * g * g;
  m[q] = mq;
  v[q] = vq;
  w[q] -= lr * (mq / c1) / (sqrtf(vq / c2) + eps);
  grad[q] = 0.f;
}

__global__ void k_to_bf16(const float* w, __nv_bfloat16* out, int np) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < np) out[q] = __float2bfloat16_rn(w[q]);
}

}  // namespace

int rank_model_params() { return H * F + H + H * H + H + H + 1; }

template <typename T>
cudaError_t launch_rank_select(const RankArgs& g, T* U, long long sU, T* Ut, long long sUt,
                               int batch, cudaStream_t st) {
  if (g.A < 1 || g.A > 128 || g.rk < 1) return cudaErrorInvalidValue;
  k_rank_select<T><<<batch, 64, 0, st>>>(g, U, sU, Ut, sUt);
  return cudaGetLastError();
}
template cudaError_t launch_rank_select<double>(const RankArgs&, double*, long long, double*,
                                                long long, int, cudaStream_t);
template cudaError_t launch_rank_select<float>(const RankArgs&, float*, long long, float*,
                                               long long, int, cudaStream_t);

cudaError_t launch_mlp_grad(const float* X, const float* tgt, const int* idx, int n, float scale,
                            const float* w, float* grad, float* loss, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_mlp_grad<<<(n + kS - 1) / kS, 256, 0, st>>>(X, tgt, idx, n, scale, w, grad, loss);
  return cudaGetLastError();
}

cudaError_t launch_adam(float* w, float* grad, float* m, float* v, int np, float lr, float b1,
                        float b2, float eps, int t, cudaStream_t st) {
  const float c1 = 1.f - powf(b1, float(t)), c2 = 1.f - powf(b2, float(t));
  k_adam<<<(np + 255) / 256, 256, 0, st>>>(w, grad, m, v, np, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

cudaError_t launch_to_bf16(const float* w, void* out, int np, cudaStream_t st) {
  k_to_bf16<<<(np + 255) / 256, 256, 0, st>>>(w, static_cast<__nv_bfloat16*>(out), np);
  return cudaGetLastError();
}

cudaError_t launch_water_fill(const double* spec, const int* cap, const int* pass_start,
                              int chi_u, int n_pass, int B, int* chi_out, float* feat,
                              cudaStream_t st) {
  if (n_pass < 1 || n_pass > 65535 || B < 1) return cudaErrorInvalidValue;
  k_water_fill<<<dim3(B, n_pass), 32, 0, st>>>(spec, cap, pass_start, chi_u, B, chi_out, feat);
  return cudaGetLastError();
}

int water_fill_max_edges() { return 32 * kWfLane; }

namespace {
__global__ void k_judge_select(const double* acc_l, const double* acc_u, const double* logz_u,
                               const int* status_u, double* logz, int* status, int* used, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const bool keep = acc_l[i] <= acc_u[i];
  if (!keep) {
    logz[i] = logz_u[i];
    status[i] = status_u[i];
  }
  used[i] = keep ? 1 : 0;
}
}  // namespace

cudaError_t launch_judge_select(const double* acc_l, const double* acc_u, const double* logz_u,
                                const int* status_u, double* logz, int* status, int* used,
                                int n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_judge_select<<<(n + 127) / 128, 128, 0, st>>>(acc_l, acc_u, logz_u, status_u, logz, status,
                                                  used, n);
  return cudaGetLastError();
}

cudaError_t launch_iota(int* x, int n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_iota<<<(n + 255) / 256, 256, 0, st>>>(x, n);
  return cudaGetLastError();
}

}  // namespace tn
