// Hutchinson estimates of the two cubic traces of the KL bound (Section 3.4):
//   tr(K~ T)  ~ (1/K) sum_k z_k^T L^T K~ L z_k
//   tr(P Kuu) ~ (1/K) sum_k z_k^T P Kuu z_k,  P Kuu z = 2 T Kuu z - T K~ T Kuu z,
// for K caller-given probe vectors z_k (M x K, row-major, entries +-1), with
// T = L L^T and K~ = Kuu + diag(s~).  Only products of the M x M matrices
// with M x K blocks are needed (O(K M^2)); all of them run in FP32 on the
// SIMT tall-skinny kernel below.
#include "common.cuh"
#include "internal.h"

namespace {

// Y[r][c] += sum_{j in this block's range} op(A)[r][j] X[j][c], plus
// d_r X[r][c] when d != null (added by the blocks of the first j range).
// op(A) = A or A^T (A: Mp x Mp FP32, entries beyond M zero).  X, Y: M x K,
// row-major, ld K.  Block: 64 rows x 64 columns of Y and a 256-long range of
// j; 256 threads, 4 x 4 outputs each; partial sums added with atomics (Y is
// zeroed first).
template <bool TRANS>
__global__ void __launch_bounds__(256) tsmm_kernel(const float* __restrict__ A, int Mp, int M,
                                                   const float* __restrict__ X, int K, const float* __restrict__ d,
                                                   float* __restrict__ Y) {
  pdl_enter();
  constexpr int JR = 256, JC = 32;
  __shared__ float As[JC][64 + 1];
  __shared__ float Xs[JC][64];
  const int r0 = blockIdx.x * 64, j0 = blockIdx.y * JR, c0 = blockIdx.z * 64;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
  const int jend = min(j0 + JR, M);
  for (int jj = j0; jj < jend; jj += JC) {
    for (int e = threadIdx.x; e < 64 * JC; e += 256) {
      int rr, jc;
      if (TRANS) { rr = e & 63; jc = e >> 6; } else { jc = e & (JC - 1); rr = e / JC; }
      const int r = r0 + rr, j = jj + jc;
      float v = 0.f;
      if (r < M && j < M) v = TRANS ? A[(size_t)j * Mp + r] : A[(size_t)r * Mp + j];
      As[jc][rr] = v;
    }
    for (int e = threadIdx.x; e < 64 * JC; e += 256) {
      const int cc = e & 63, jc = e >> 6;
      const int c = c0 + cc, j = jj + jc;
      Xs[jc][cc] = (c < K && j < M) ? X[(size_t)j * K + c] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int jc = 0; jc < JC; ++jc) {
      float av[4], xv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[jc][ty * 4 + a];
#pragma unroll
      for (int b = 0; b < 4; ++b) xv[b] = Xs[jc][tx * 4 + b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(av[a], xv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int r = r0 + ty * 4 + a;
    if (r >= M) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int c = c0 + tx * 4 + b;
      if (c >= K) continue;
      float v = acc[a][b];
      if (d && blockIdx.y == 0) v = fmaf(d[r], X[(size_t)r * K + c], v);
      atomicAdd(Y + (size_t)r * K + c, v);
    }
  }
}

// *dst += sum_e U_e V_e (n elements, FP64 accumulation per block).
__global__ void dot_kernel(const float* __restrict__ U, const float* __restrict__ V, size_t n, double* dst) {
  pdl_enter();
  double part = 0.0;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    part += (double)U[e] * (double)V[e];
  block_add_double(part, dst);
}

void tsmm(const float* A, int Mp, int M, bool trans, const float* X, int K, const float* d, float* Y,
          cudaStream_t st) {
  k_zero(st, Y, sizeof(float) * (size_t)M * K);
  dim3 grid((M + 63) / 64, (M + 255) / 256, (K + 63) / 64);
  svgp_note_launch();
  if (trans) pdl_launch(tsmm_kernel<true>, grid, 256, 0, st, A, Mp, M, X, K, d, Y);
  else pdl_launch(tsmm_kernel<false>, grid, 256, 0, st, A, Mp, M, X, K, d, Y);
}

void dot(const float* U, const float* V, size_t n, double* dst, cudaStream_t st) {
  int grid = (int)((n + 255) / 256);
  if (grid > 256) grid = 256;
  svgp_note_launch();
  pdl_launch(dot_kernel, grid, 256, 0, st, U, V, n, dst);
}

}  // namespace

void k_hutchinson(const float* Lf, const float* Kuu, const float* s, int M, int Mp, const float* Z, int K,
                  float* bufA, float* bufB, float* bufC, double* red, cudaStream_t st) {
  const size_t n = (size_t)M * K;
  // tr(K~ T): A = L Z, B = K~ A, <A, B>
  tsmm(Lf, Mp, M, false, Z, K, nullptr, bufA, st);
  tsmm(Kuu, Mp, M, false, bufA, K, s, bufB, st);
  dot(bufA, bufB, n, red + RED_HKT, st);
  // tr(P Kuu): A = Kuu Z, B = L^T A, A = L B (= T Kuu Z), <Z, A>;
  // B = K~ A, C = L^T B, B = L C (= T K~ T Kuu Z), <Z, B>
  tsmm(Kuu, Mp, M, false, Z, K, nullptr, bufA, st);
  tsmm(Lf, Mp, M, true, bufA, K, nullptr, bufB, st);
  tsmm(Lf, Mp, M, false, bufB, K, nullptr, bufA, st);
  dot(Z, bufA, n, red + RED_HW1, st);
  tsmm(Kuu, Mp, M, false, bufA, K, s, bufB, st);
  tsmm(Lf, Mp, M, true, bufB, K, nullptr, bufC, st);
  tsmm(Lf, Mp, M, false, bufC, K, nullptr, bufB, st);
  dot(Z, bufB, n, red + RED_HX4, st);
}
