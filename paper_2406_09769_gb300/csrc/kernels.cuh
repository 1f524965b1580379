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
cudaError_t launch_eigh_top(const T* L, long long sL, double* U, long long sU, double* lam,
                            long long slam, int n, int r, int nlam, int* status, int batch,
                            cudaStream_t st);
template <typename T>
size_t eigh_smem_bytes(int n, int r, int nlam);
template <typename T>
size_t eigh_smem_limit();
cudaError_t eigh_configure();

}  // namespace tn
