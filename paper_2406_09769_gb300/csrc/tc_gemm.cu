// Batched tensor-core contraction for sm_103a (tcgen05 + TMA + TMEM).
//
//   C_i[m][n] = alpha_i * sum_k A_i[m][k] * B_i[n][k]      i = 0 .. batch-1
//
// A (M x K) and B (N x K) are row-major FP32 with K contiguous ("K-major"),
// X_i = X + i * sX.  Every density-matrix contraction of the method is cast in
// this form (B = R is symmetric; transposed copies are written where needed).
//
// One CTA of 256 threads computes a 128 x BN tile (BN <= 256, multiple of 16):
//   * thread 0 streams 32-wide K chunks of A and B into 128B-swizzled shared
//     memory with 3D TMA loads (batch = third dimension; out-of-range rows,
//     columns and K are zero-filled by TMA), through a ring of up to four
//     stages guarded by mbarriers (all chunks of a K = 128 contraction in
//     flight at once);
//   * thread 0 issues tcgen05.mma.cta_group::1.kind::tf32 (M = 128, N = BN,
//     K = 8 per instruction), accumulating in TMEM (128 lanes x BN columns),
//     and tcgen05.commit releases each stage;
//   * with `split`, every staged tile is split into x = hi + lo (hi = x
//     rounded to TF32, in place; lo into one of two buffers of its own) and
//     three products hi*hi + hi*lo + lo*hi are accumulated: the compensated
//     pass of the value path (~FP32 accuracy);
//   * the eight warps read TMEM (warp w: lanes 32 (w % 4) .., alternate
//     16-column groups) with tcgen05.ld.32x32b, scale, and store C (row-major)
//     and/or C^T, folding max|C| into an atomic slot.
// Every mbarrier wait is bounded; on expiry the kernel sets *err, waits
// (bounded) for its own TMA copies, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "kernels.cuh"

namespace tn {

namespace {

constexpr int kTcThreads = 256;
constexpr int kLoBufs = 1;                    // lo halves of split chunks in flight
constexpr uint32_t kEpiBytes = 8 * 32 * 33 * 4;  // per-warp 32 x 32 transpose tiles (padded)
constexpr int kChunk = 32;                    // K elements per stage (128 bytes of FP32)
constexpr uint32_t kWaitLimit = 1u << 22;     // bounded spin on every mbarrier
constexpr uint32_t kPollLimit = 1u << 14;     // bounded poll of TcGemmArgs::poll

__device__ __forceinline__ uint32_t su32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity) {
  for (uint32_t i = 0; i < kWaitLimit; ++i)
    if (mbar_try(b, parity)) return true;
  return false;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0,
                                            int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(su32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(su32(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128B swizzle, rows of 128 B,
// 8-row groups 1024 B apart (stride byte offset), fixed version bits 46..48 = 1.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= uint64_t((saddr >> 4) & 0x3FFFu);
  d |= uint64_t(1) << 16;                 // leading byte offset (unused for swizzled K-major)
  d |= uint64_t(1024 >> 4) << 32;         // stride byte offset
  d |= uint64_t(1) << 46;                 // descriptor version
  d |= uint64_t(2) << 61;                 // SWIZZLE_128B
  return d;
}

// Instruction descriptor, kind::tf32: D = F32, A = B = TF32, both K-major.
__host__ __device__ __forceinline__ uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

__device__ __forceinline__ void umma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                          uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ float tf32_hi(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

struct SmemPlan {
  uint32_t a_bytes, b_bytes, stage_bytes, stages, split;
};

__global__ void __launch_bounds__(kTcThreads) k_tc_gemm(const __grid_constant__ CUtensorMap tmA,
                                                      const __grid_constant__ CUtensorMap tmB,
                                                      TcGemmArgs g, int BN, int stages,
                                                      uint32_t tmem_cols) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte alignment of the stage ring (required by the 128B swizzle atoms)
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t a_bytes = 128 * 128;
  const uint32_t b_bytes = uint32_t(BN) * 128;
  const uint32_t tile_bytes = a_bytes + b_bytes;
  const int nlo = g.split ? kLoBufs : 0;
  unsigned char* lo_base = base + stages * tile_bytes;
  uint32_t region = (stages + nlo) * tile_bytes;  // the epilogue reuses it for transposes
  if (region < kEpiBytes) region = kEpiBytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(base + region);
  uint64_t* freed = full + stages;
  uint64_t* lofree = freed + stages;   // kLoBufs
  uint64_t* done = lofree + kLoBufs;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n0 = blockIdx.x * BN, m0 = blockIdx.y * 128, bi = blockIdx.z;
  const int nk = (g.K + kChunk - 1) / kChunk;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(tmem_slot)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&freed[s], 1);
    }
    for (int q = 0; q < kLoBufs; ++q) mbar_init(&lofree[q], 1);
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = idesc_tf32(128, BN);

  // Every chunk's TMA is issued as early as its stage allows: all of them up
  // front when the ring holds the whole K extent; otherwise the stage of chunk
  // kc - 1 is refilled right after chunk kc's MMAs are issued (its own MMAs,
  // issued one chunk earlier, have usually completed by then).  With `split`
  // the lo halves go to kLoBufs buffers of their own, so a stage is released
  // by the MMAs alone and loads overlap the split of later chunks.
  int issued = 0;    // chunks whose TMA has been issued (thread 0)
  int consumed = 0;  // chunks whose arrival thread 0 has observed
  auto issue = [&](int kc) {
    const int s = kc % stages;
    unsigned char* st = base + s * tile_bytes;
    mbar_expect_tx(&full[s], tile_bytes);
    tma_load_3d(st, &tmA, &full[s], kc * kChunk, m0, bi);
    tma_load_3d(st + a_bytes, &tmB, &full[s], kc * kChunk, n0, bi);
  };
  if (tid == 0) {
    for (; issued < nk && issued < stages; ++issued) issue(issued);
  }
  // A bounded wait on a device flag that nothing sets, when the caller asks
  // for it: its expiry takes the same path as an expired mbarrier wait
  // (error flag, drain of the TMA copies in flight, TMEM released).
  if (tid == 0 && g.poll) {
    bool seen = false;
    for (uint32_t i = 0; i < kPollLimit && !seen; ++i)
      seen = *reinterpret_cast<const volatile int*>(g.poll) != 0;
    if (!seen) *abort_flag = 1;
  }
  __syncthreads();
  const int nk_run = *abort_flag ? 0 : nk;
  int mma_chunks = 0;  // chunks whose MMAs thread 0 has issued
  for (int kc = 0; kc < nk_run; ++kc) {
    const int s = kc % stages;
    const uint32_t ph = uint32_t(kc / stages) & 1u;
    unsigned char* st = base + s * tile_bytes;
    unsigned char* lo = lo_base + (kc % kLoBufs) * tile_bytes;
    if (g.split) {
      // every thread: the chunk has landed and its lo buffer is free (the
      // MMAs of chunk kc - kLoBufs have completed); then split in place
      bool ok = mbar_wait(&full[s], ph);
      if (ok && kc >= kLoBufs)
        ok = mbar_wait(&lofree[kc % kLoBufs], uint32_t(kc / kLoBufs - 1) & 1u);
      if (!ok) atomicExch(abort_flag, 1);
      if (tid == 0 && ok) consumed = kc + 1;
      __syncthreads();
      if (*abort_flag) break;
      float4* hi = reinterpret_cast<float4*>(st);
      float4* lq = reinterpret_cast<float4*>(lo);
      for (uint32_t q = tid; q < tile_bytes / 16; q += kTcThreads) {
        const float4 x = hi[q];
        const float4 h = make_float4(tf32_hi(x.x), tf32_hi(x.y), tf32_hi(x.z), tf32_hi(x.w));
        hi[q] = h;
        lq[q] = make_float4(x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
    }
    if (tid == 0) {
      bool ok = true;
      if (!g.split) {
        ok = mbar_wait(&full[s], ph);
        if (ok) consumed = kc + 1;
        else *abort_flag = 1;
      }
      if (ok) {
        tc_fence_after();
        const uint32_t a0 = su32(st), b0 = su32(st + a_bytes);
        const uint32_t al0 = su32(lo), bl0 = su32(lo + a_bytes);
        for (int j = 0; j < kChunk / 8; ++j) {
          const uint32_t acc = (kc > 0 || j > 0) ? 1u : 0u;
          const uint64_t ah = desc_sw128(a0 + 32 * j), bh = desc_sw128(b0 + 32 * j);
          umma_tf32(tmem, ah, bh, idesc, acc);
          if (g.split) {
            umma_tf32(tmem, ah, desc_sw128(bl0 + 32 * j), idesc, 1u);
            umma_tf32(tmem, desc_sw128(al0 + 32 * j), bh, idesc, 1u);
          }
        }
        umma_commit(&freed[s]);
        if (g.split) umma_commit(&lofree[kc % kLoBufs]);
        mma_chunks = kc + 1;
        // refill the stage of chunk kc - 1 (of chunk kc itself with a single
        // stage) with the next chunk
        const int pc = (stages > 1) ? kc - 1 : kc;
        if (pc >= 0 && issued < nk) {
          if (mbar_wait(&freed[pc % stages], uint32_t(pc / stages) & 1u)) {
            issue(issued);
            ++issued;
          } else {
            *abort_flag = 1;
          }
        }
      }
    }
    if (!g.split && tid == 0 && *abort_flag) break;  // thread 0 alone runs the non-split loop
  }
  // every MMA issued so far has completed before TMEM is read or released
  if (tid == 0) umma_commit(done);
  __syncthreads();
  bool good = (*abort_flag == 0) && (mma_chunks == nk || tid != 0);
  if (!mbar_wait(done, 0)) good = false;
  if (!__syncthreads_and(good)) {
    good = false;
    if (tid == 0) {
      atomicExch(g.err, 1);
      // drain: TMA chunks still in flight must land before the CTA exits
      for (int kc = consumed; kc < issued; ++kc)
        mbar_wait(&full[kc % stages], uint32_t(kc / stages) & 1u);
    }
  }
  __syncthreads();
  tc_fence_after();
  if (good) {
    float alpha = 1.f;
    if (g.amax_in) {
      const float mx = __uint_as_float(g.amax_in[(long long)bi * g.s_amax_in]);
      alpha = (mx > 0.f) ? 1.f / mx : 1.f;
    }
    // warp w reads TMEM lanes 32 (w % 4) .. + 31 (one row each) and every other
    // 32-column group; C^T is stored from there (lanes = rows run along C^T's
    // rows), C after a transpose through a per-warp shared tile (lanes =
    // columns, 128-byte rows).  TMEM holds at least round_up(BN, 32) columns.
    const int rbase = m0 + (warp & 3) * 32;
    const int gm = rbase + lane;
    float* tile = reinterpret_cast<float*>(base) + warp * (32 * 33);
    float lmax = 0.f;
    bool bad = false;
    for (int c0 = 32 * (warp >> 2); c0 < BN; c0 += 64) {
      uint32_t v[32];
      const uint32_t taddr = tmem + (uint32_t((warp & 3) * 32) << 16) + uint32_t(c0);
      tmem_ld16(taddr, *reinterpret_cast<uint32_t(*)[16]>(&v[0]));
      tmem_ld16(taddr + 16, *reinterpret_cast<uint32_t(*)[16]>(&v[16]));
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int gn = n0 + c0 + j;
        const float x = alpha * __uint_as_float(v[j]);
        tile[lane * 33 + j] = x;
        if (gm < g.M && gn < g.N) {
          if (g.Ct) {
            const int q = gn / g.ct_cols, cc = gn - q * g.ct_cols;
            g.Ct[(long long)bi * g.sCt + (long long)cc * g.ldct + (long long)gm * (g.N / g.ct_cols) + q] = x;
          }
          lmax = fmaxf(lmax, fabsf(x));
          bad |= !isfinite(x);
        }
      }
      __syncwarp();
      if (g.C) {
        const int gn = n0 + c0 + lane;
        if (gn < g.N) {
          float* Cb = g.C + (long long)bi * g.sC + gn;
          for (int i = 0; i < 32 && rbase + i < g.M; ++i)
            Cb[(long long)(rbase + i) * g.ldc] = tile[i * 33 + lane];
        }
      }
      __syncwarp();
    }
    if (g.amax_out) {
      if (bad) lmax = INFINITY;
      for (int o = 16; o > 0; o >>= 1) lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
      if (lane == 0) atomicMax(g.amax_out + (long long)bi * g.s_amax_out, __float_as_uint(lmax));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols)
                 : "memory");
  }
}

// ---------------------------------------------------------------- host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

bool make_map(CUtensorMap* m, const float* ptr, int K, int rows, int batch, long long ld,
              long long sBatch, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {cuuint64_t(K), cuuint64_t(rows), cuuint64_t(batch)};
  cuuint64_t strides[2] = {cuuint64_t(ld) * 4, cuuint64_t(sBatch) * 4};
  cuuint32_t box[3] = {uint32_t(kChunk), uint32_t(box_rows), 1};
  cuuint32_t estr[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(ptr), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

size_t tc_gemm_smem_bytes(int BN, int split, int K, int* stages_out, int budget_kb) {
  // A ring of K-chunk stages (TMA targets), up to 4 and no more than the K
  // chunks, plus kLoBufs buffers for the lo halves of split chunks, within
  // the budget (default ~104 KB, so that two CTAs share an SM: one CTA's
  // loads and epilogue overlap the other's MMAs; the autotuner also tries
  // other budgets and tile widths per contraction shape).
  const size_t tile = size_t(128 + BN) * 128;
  const size_t lo = split ? kLoBufs * tile : 0;
  const size_t budget = size_t(budget_kb > 0 ? budget_kb : 104) * 1024;
  int stages = budget > lo ? int((budget - lo) / tile) : 1;
  const int nk = (K + kChunk - 1) / kChunk;
  if (stages > nk) stages = nk;
  if (stages > 4) stages = 4;
  if (stages < 1) stages = 1;
  if (stages_out) *stages_out = stages;
  size_t region = stages * tile + lo;
  if (region < kEpiBytes) region = kEpiBytes;
  return 1024 + region + (2 * stages + kLoBufs + 1) * 8 + 16;
}

cudaError_t tc_gemm_configure() {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  if (!encode_fn()) return cudaErrorNotSupported;
  return cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
}

cudaError_t launch_tc_gemm(const TcGemmArgs& g, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return cudaSuccess;
  if (g.Ct && (g.ct_cols <= 0 || g.N % g.ct_cols)) return cudaErrorInvalidValue;
  if (g.K <= 0 || (g.lda % 4) || (g.ldb % 4) || (g.sA % 4) || (g.sB % 4) ||
      (reinterpret_cast<uintptr_t>(g.A) % 16) || (reinterpret_cast<uintptr_t>(g.B) % 16))
    return cudaErrorInvalidValue;
  int BN = ((g.N + 15) / 16) * 16;
  if (BN > 256) BN = 256;
  if (g.bn > 0) {
    if (g.bn % 16 || g.bn > 256) return cudaErrorInvalidValue;
    BN = g.bn;
  }
  CUtensorMap ma, mb;
  if (!make_map(&ma, g.A, g.K, g.M, g.batch, g.lda, g.sA, 128)) return cudaErrorInvalidValue;
  if (!make_map(&mb, g.B, g.K, g.N, g.batch, g.ldb, g.sB, BN)) return cudaErrorInvalidValue;
  int stages = 1;
  const size_t smem = tc_gemm_smem_bytes(BN, g.split, g.K, &stages, g.budget_kb);
  uint32_t cols = 32;
  while (cols < uint32_t(BN)) cols <<= 1;
  dim3 grid((g.N + BN - 1) / BN, (g.M + 127) / 128, g.batch);
  k_tc_gemm<<<grid, kTcThreads, smem, st>>>(ma, mb, g, BN, stages, cols);
  return cudaGetLastError();
}

}  // namespace tn
