// Arithmetic peaks of this device, measured by short burst kernels, for the
// roofline denominators of the kernels that are not bandwidth bound: the FP32
// pipe (the eigensolver, SVD and Cholesky), the FP64 pipe (the FP64 path) and
// the tcgen05 tensor pipe in kind::tf32 (the mixed path's contractions).
//
//   FP32 / FP64: every thread runs 16 independent FMA chains (FP32 also as
//   packed FP32x2), a multiple of the SM count in CTAs of 256 threads;
//   TF32: one thread per CTA issues tcgen05.mma kind::tf32, M = 128, N = 256,
//   K = 8, from small nonzero shared-memory operands into one TMEM accumulator,
//   back to back; two CTAs per SM (256 TMEM columns each).  Each burst is
//   timed with CUDA events; the best of three is kept.
// Every mbarrier wait is bounded; on expiry the kernel records an error,
// waits once more (bounded) for its MMAs, frees its TMEM and returns.
#include <cuda_runtime.h>

#include <cstdint>

#include "tn_dmtree.h"

namespace {

constexpr int kIters = 4096;

__global__ void __launch_bounds__(256) k_peak_ffma(const float* __restrict__ in, float* out) {
  const float m = in[0], c = in[1];
  float a[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) a[i] = in[2] + float(i) * 1e-3f + float(threadIdx.x) * 1e-6f;
  for (int it = 0; it < kIters; ++it)
#pragma unroll
    for (int i = 0; i < 16; ++i) a[i] = fmaf(a[i], m, c);
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < 16; ++i) s += a[i];
  if (s == 12345.f) out[blockIdx.x] = s;  // keeps the chains live
}

__global__ void __launch_bounds__(256) k_peak_ffma2(const float* __restrict__ in, float* out) {
  const float2 m = make_float2(in[0], in[0]), c = make_float2(in[1], in[1]);
  float2 a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
    a[i] = make_float2(in[2] + float(i) * 1e-3f, in[2] + float(threadIdx.x) * 1e-6f);
  for (int it = 0; it < kIters; ++it)
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = __ffma2_rn(a[i], m, c);
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += a[i].x + a[i].y;
  if (s == 12345.f) out[blockIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_peak_dfma(const double* __restrict__ in, double* out) {
  const double m = in[0], c = in[1];
  double a[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) a[i] = in[2] + double(i) * 1e-3 + double(threadIdx.x) * 1e-6;
  for (int it = 0; it < kIters / 8; ++it)
#pragma unroll
    for (int i = 0; i < 16; ++i) a[i] = fma(a[i], m, c);
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 16; ++i) s += a[i];
  if (s == 12345.0) out[blockIdx.x] = s;
}

// ------------------------------------------------------------------ TF32
constexpr uint32_t kMmaWaitLimit = 1u << 24;
constexpr int kMmaIters = 2048;  // groups of four K = 8 instructions (one 128-byte row)

__device__ __forceinline__ uint32_t su32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// K-major operand, 128-byte swizzle, 128-byte rows, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= uint64_t((saddr >> 4) & 0x3FFFu);
  d |= uint64_t(1) << 16;
  d |= uint64_t(1024 >> 4) << 32;
  d |= uint64_t(1) << 46;
  d |= uint64_t(2) << 61;
  return d;
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
  for (uint32_t i = 0; i < kMmaWaitLimit; ++i)
    if (mbar_try(b, parity)) return true;
  return false;
}

__global__ void __launch_bounds__(128) k_peak_tf32(int* err) {
  extern __shared__ __align__(1024) unsigned char raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
  unsigned char* A = base;               // 128 rows x 128 B
  unsigned char* B = base + 128 * 128;   // 256 rows x 128 B
  uint64_t* done = reinterpret_cast<uint64_t*>(B + 256 * 128);
  uint32_t* slot = reinterpret_cast<uint32_t*>(done + 1);
  const int tid = threadIdx.x;
  for (int i = tid; i < (128 + 256) * 128 / 4; i += blockDim.x)  // small nonzero operands
    reinterpret_cast<float*>(base)[i] = float((i * 13) % 17) * 0.0625f;
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(slot)),
                 "r"(256u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(done)), "r"(1u) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // operands visible to tcgen05
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *slot;
  bool ok = true;
  if (tid == 0) {
    // D = F32, A = B = TF32, K-major, M = 128, N = 256
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(256 >> 3) << 17) |
                           (uint32_t(128 >> 4) << 24);
    const uint32_t a0 = su32(A), b0 = su32(B);
    for (int it = 0; it < kMmaIters; ++it)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint64_t ad = desc_sw128(a0 + 32 * j), bd = desc_sw128(b0 + 32 * j);
        const uint32_t acc = (it | j) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            su32(done))
        : "memory");
    if (!mbar_wait(done, 0)) {
      atomicExch(err, 1);
      ok = mbar_wait(done, 0);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  (void)ok;
  if (tid < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256u)
                 : "memory");
}

template <class F>
float best_ms(F&& launch, cudaEvent_t e0, cudaEvent_t e1, cudaError_t* e) {
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {  // the first launch warms up
    *e = cudaEventRecord(e0);
    if (*e != cudaSuccess) return best;
    launch();
    *e = cudaGetLastError();
    if (*e != cudaSuccess) return best;
    *e = cudaEventRecord(e1);
    if (*e != cudaSuccess) return best;
    *e = cudaEventSynchronize(e1);
    if (*e != cudaSuccess) return best;
    float ms = 0.f;
    *e = cudaEventElapsedTime(&ms, e0, e1);
    if (*e != cudaSuccess) return best;
    if (rep > 0 && ms < best) best = ms;
  }
  return best;
}

}  // namespace

extern "C" tn_status tn_measure_peaks(int32_t device, double* tflops) {
  if (!tflops) return TN_ERR_INVALID;
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return TN_ERR_CUDA;
  int sms = 0, major = 0, minor = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device);
  if (sms < 1) return TN_ERR_CUDA;
  float* fin = nullptr;
  int* err = nullptr;
  if (cudaMalloc(&fin, 64 * sizeof(double) + 1024 * 1024) != cudaSuccess) {
    cudaGetLastError();
    return TN_ERR_OOM;
  }
  if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(fin);
    return TN_ERR_OOM;
  }
  const float hf[3] = {0.999f, 1e-3f, 0.5f};
  const double hd[3] = {0.999, 1e-3, 0.5};
  cudaMemcpy(fin, hf, sizeof(hf), cudaMemcpyHostToDevice);
  double* din = reinterpret_cast<double*>(fin + 16);
  cudaMemcpy(din, hd, sizeof(hd), cudaMemcpyHostToDevice);
  cudaMemset(err, 0, sizeof(int));
  float* fout = fin + 64;
  double* dout = reinterpret_cast<double*>(fin + 64);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int grid = sms * 8;
  const double threads = double(grid) * 256.0;
  tn_status st = TN_OK;
  const float ms_f = best_ms([&] { k_peak_ffma<<<grid, 256>>>(fin, fout); }, e0, e1, &e);
  if (e == cudaSuccess) tflops[0] = threads * 16.0 * kIters * 2.0 / (ms_f * 1e-3) / 1e12;
  const float ms_f2 = best_ms([&] { k_peak_ffma2<<<grid, 256>>>(fin, fout); }, e0, e1, &e);
  if (e == cudaSuccess) tflops[1] = threads * 16.0 * kIters * 2.0 / (ms_f2 * 1e-3) / 1e12;
  const float ms_d = best_ms([&] { k_peak_dfma<<<grid, 256>>>(din, dout); }, e0, e1, &e);
  if (e == cudaSuccess) tflops[2] = threads * 16.0 * (kIters / 8) * 2.0 / (ms_d * 1e-3) / 1e12;
  tflops[3] = 0.0;
  if (e == cudaSuccess && major == 10 && minor == 3) {
    const size_t smem = 1024 + (128 + 256) * 128 + 64;
    e = cudaFuncSetAttribute(k_peak_tf32, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e == cudaSuccess) {
      const int tgrid = sms * 2;
      const float ms_t = best_ms([&] { k_peak_tf32<<<tgrid, 128, smem>>>(err); }, e0, e1, &e);
      int herr = 0;
      if (e == cudaSuccess) e = cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
      if (e == cudaSuccess && !herr)
        tflops[3] = double(tgrid) * kMmaIters * 4.0 * (2.0 * 128 * 256 * 8) / (ms_t * 1e-3) / 1e12;
      else if (herr)
        st = TN_ERR_TIMEOUT;
    }
  }
  if (e != cudaSuccess) st = TN_ERR_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(fin);
  cudaFree(err);
  cudaGetLastError();
  return st;
}
