// Blocks of general plans: every chain position's tensors contracted together
// ("contract T(v) first", Sec. 5.3), with a delta for every edge passing
// through the position, by a short program of gather-contractions (pairwise
// products into scratch, then one op writing the block).  One thread per
// output element; the summed slots run as a mixed-radix counter.  The blocks
// are small next to the density-matrix work (a few MB per pass), so the
// kernel favours generality: operands are read through the L1/L2 caches.
#include "kernels.cuh"

namespace tn {
namespace {

constexpr int kMaxSlots = 48;
constexpr int kThreads = 256;

// The elements of ops [a, b) of one instance: raw site tensors at raw (times
// iv), previous MPS sites at Si, scratch at sc, blocks at Yi (and Yti).
template <typename TS, typename TY>
__device__ __forceinline__ void gather_range(const GOp* __restrict__ ops,
                                             const GTen* __restrict__ ten,
                                             const int32_t* __restrict__ code,
                                             const int64_t* __restrict__ pre, int a, int b,
                                             const double* raw, const double* iv, const TS* Si,
                                             double* sc, TY* Yi, TY* Yti,
                                             const GuardTab* gd = nullptr) {
  if (!guard_ok(gd, pre + a, 8, 0x301) || !guard_ok(gd, pre + b, 8, 0x301)) return;
  const int64_t e0 = pre[a], e1 = pre[b];
  for (int64_t e = e0 + int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < e1;
       e += int64_t(gridDim.x) * blockDim.x) {
    int lo = a, hi = b - 1;  // the op holding element e: last i with pre[i] <= e
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (pre[mid] <= e) lo = mid;
      else hi = mid - 1;
    }
    if (!guard_ok(gd, ops + lo, sizeof(GOp), 0x302)) continue;
    const GOp op = ops[lo];
    const int64_t idx = e - pre[lo];
    const int32_t* sdim = code + op.code_off;
    const int32_t* oslot = sdim + op.ns;
    const int32_t* sslot = oslot + op.nout;
    if (gd && (!guard_idx(gd, op.ns, kMaxSlots + 1, 0x303) ||
               !guard_ok(gd, sdim, 4ll * (op.ns + op.nout + op.nsum), 0x304)))
      continue;
    int val[kMaxSlots];
    for (int s = 0; s < op.ns; ++s) val[s] = -1;
    bool ok = true;
    int64_t rem = idx;
    for (int i = op.nout - 1; i >= 0; --i) {
      const int s = oslot[i];
      if (!guard_idx(gd, s, op.ns, 0x305)) { ok = false; break; }
      const int dv = sdim[s];
      const int v = int(rem % dv);
      rem /= dv;
      if (val[s] >= 0 && val[s] != v) ok = false;
      val[s] = v;
    }
    double acc = 0.0;
    if (ok && gd)
      for (int i = 0; i < op.nsum; ++i)
        if (!guard_idx(gd, sslot[i], op.ns, 0x306)) ok = false;
    if (ok) {
      for (int i = 0; i < op.nsum; ++i) val[sslot[i]] = 0;
      while (true) {
        double prod = 1.0;
        for (int t = 0; t < op.nt; ++t) {
          if (!guard_ok(gd, ten + op.t_first + t, sizeof(GTen), 0x307)) { prod = 0.0; break; }
          const GTen g = ten[op.t_first + t];
          const int32_t* lg = code + g.leg_off;
          int64_t off = g.base;
          bool lok = true;
          for (int j = 0; j < g.nleg; ++j) {
            if (gd && !guard_idx(gd, lg[2 * j], op.ns, 0x308)) { lok = false; break; }
            off += int64_t(val[lg[2 * j]]) * lg[2 * j + 1];
          }
          double x = 0.0;
          if (!lok) {
          } else if (g.src == 0) {
            if (guard_ok(gd, raw + off, 8, 0x309) && guard_ok(gd, iv + g.vertex, 8, 0x30a))
              x = raw[off] * iv[g.vertex];
          } else if (g.src == 1) {
            if (guard_ok(gd, Si + off, sizeof(TS), 0x30b)) x = double(Si[off]);
          } else {
            if (guard_ok(gd, sc + off, 8, 0x30c)) x = sc[off];
          }
          prod *= x;
        }
        acc += prod;
        int i = 0;
        for (; i < op.nsum; ++i) {
          const int s = sslot[i];
          if (++val[s] < sdim[s]) break;
          val[s] = 0;
        }
        if (i == op.nsum) break;
      }
    }
    if (op.to_block) {
      if (guard_ok(gd, Yi + op.dst_off + idx, sizeof(TY), 0x30d)) Yi[op.dst_off + idx] = TY(acc);
      if (Yti) {
        const int64_t l = idx / op.dkDr, j = idx - l * op.dkDr;
        if (guard_ok(gd, Yti + op.dst_off + j * op.Dl + l, sizeof(TY), 0x30e))
          Yti[op.dst_off + j * op.Dl + l] = TY(acc);
      }
    } else {
      if (guard_ok(gd, sc + op.dst_off + idx, 8, 0x30f)) sc[op.dst_off + idx] = acc;
    }
  }
}

template <typename TS, typename TY>
__global__ void __launch_bounds__(kThreads)
    k_gather(const GOp* __restrict__ ops, const GTen* __restrict__ ten,
             const int32_t* __restrict__ code, const int64_t* __restrict__ pre, int a, int b,
             const double* const* __restrict__ tens, const double* __restrict__ inv,
             long long sInv, const TS* __restrict__ S, long long sS, double* scr, long long sScr,
             TY* __restrict__ Y, long long sY, TY* __restrict__ Yt) {
  const int inst = blockIdx.y;
  gather_range<TS, TY>(ops, ten, code, pre, a, b, tens[inst], inv + inst * sInv,
                       S ? S + inst * sS : nullptr, scr ? scr + inst * sScr : nullptr,
                       Y + inst * sY, Yt ? Yt + inst * sY : nullptr);
}

// grouped: blockIdx.y = problem (one instance of one bucket at one level);
// kGuard: the range guard checked on every global access
template <bool kGuard>
__global__ void __launch_bounds__(kThreads) k_gather_grouped(const GatherDesc* __restrict__ desc) {
  const GatherDesc q = desc[blockIdx.y];
  gather_range<float, float>(q.ops, q.ten, q.code, q.pre, q.a, q.b, q.raw, q.inv, q.S, q.scr, q.Y,
                             q.Yt, kGuard ? q.guard : nullptr);
}

}  // namespace

template <typename TS, typename TY>
cudaError_t launch_gather(const GOp* ops, const GTen* ten, const int32_t* code, const int64_t* pre,
                          int a, int b, int64_t n_elems, const double* const* tens,
                          const double* inv, long long sInv, const TS* S, long long sS,
                          double* scr, long long sScr, TY* Y, long long sY, TY* Yt, int batch,
                          cudaStream_t st) {
  if (b <= a || n_elems <= 0) return cudaSuccess;
  const int64_t want = (n_elems + kThreads - 1) / kThreads;
  const int grid = int(want < 152 * 8 ? want : 152 * 8);
  k_gather<TS, TY><<<dim3(grid, batch), kThreads, 0, st>>>(ops, ten, code, pre, a, b, tens, inv,
                                                           sInv, S, sS, scr, sScr, Y, sY, Yt);
  return cudaGetLastError();
}

cudaError_t launch_gather_grouped(const GatherDesc* desc, int n_prob, int64_t max_elems,
                                  bool guarded, cudaStream_t st) {
  if (n_prob <= 0 || max_elems <= 0) return cudaSuccess;
  if (n_prob > 65535) return cudaErrorInvalidValue;
  const int64_t want = (max_elems + kThreads - 1) / kThreads;
  const int grid = int(want < 64 ? want : 64);
  if (guarded) k_gather_grouped<true><<<dim3(grid, n_prob), kThreads, 0, st>>>(desc);
  else k_gather_grouped<false><<<dim3(grid, n_prob), kThreads, 0, st>>>(desc);
  return cudaGetLastError();
}

template cudaError_t launch_gather<double, double>(const GOp*, const GTen*, const int32_t*,
                                                   const int64_t*, int, int, int64_t,
                                                   const double* const*, const double*, long long,
                                                   const double*, long long, double*, long long,
                                                   double*, long long, double*, int, cudaStream_t);
template cudaError_t launch_gather<float, float>(const GOp*, const GTen*, const int32_t*,
                                                 const int64_t*, int, int, int64_t,
                                                 const double* const*, const double*, long long,
                                                 const float*, long long, double*, long long,
                                                 float*, long long, float*, int, cudaStream_t);

}  // namespace tn
