// Hutchinson estimates of the two cubic traces of the KL bound (Section 3.4):
//   tr(K~ T)  ~ (1/K) sum_k z_k^T L^T K~ L z_k
//   tr(P Kuu) ~ (1/K) sum_k z_k^T P Kuu z_k,  P Kuu z = 2 T Kuu z - T K~ T Kuu z,
// for K caller-given probe vectors z_k (M x K, row-major, entries +-1), with
// T = L L^T and K~ = Kuu + diag(s~).  Only products of the M x M matrices
// with M x K blocks are needed (O(K M^2)); all of them run in FP32 on the
// SIMT tall-skinny kernel below.
//
// The rest of the bound without P = 2T - T K~ T (so without the O(M^3)
// chain): per point, with u = L^T k_n and w = L u = T k_n,
//   k_n^T P k_n = 2 u^T u - w^T K~ w,
// over the columns of Kuf in blocks of up to 256 points (O(B M^2)); and
// v = P m~ = 2 T m~ - T K~ T m~ by the same products on one column.
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

// Kuf[i][c] = sf2 exp(-1/2 |z~_i - x~_{c0+c}|^2) for c < nc (FP32, scaled
// coordinates Zs, Xs with Dp floats per point), row-major with ld nc.
__global__ void kuf_dense_kernel(const float* __restrict__ Zs, const float* __restrict__ Xs, int M, int D,
                                 const float* __restrict__ sf2, int c0, int nc, float* __restrict__ out) {
  pdl_enter();
  const int Dp = (D + 3) & ~3;
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)M * nc) return;
  const int i = (int)(e / nc), c = (int)(e % nc);
  const float* z = Zs + (size_t)i * Dp;
  const float* x = Xs + (size_t)(c0 + c) * Dp;
  float d2 = 0.f;
  for (int d = 0; d < D; ++d) {
    const float t = __ldg(z + d) - __ldg(x + d);
    d2 = fmaf(t, t, d2);
  }
  out[e] = *sf2 * expf(-0.5f * d2);
}

// q_c = 2 sum_i U[i][c]^2 - sum_i W[i][c] V[i][c] (= k^T P k of column c) into
// q[c] and, summed, into *dst.  One thread per column (coalesced rows).
__global__ void colq_kernel(const float* __restrict__ U, const float* __restrict__ W, const float* __restrict__ V,
                            int M, int nc, float* __restrict__ q, double* dst) {
  pdl_enter();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  double part = 0.0;
  if (c < nc) {
    float a = 0.f, b = 0.f;
    for (int i = 0; i < M; ++i) {
      const size_t e = (size_t)i * nc + c;
      const float u = U[e];
      a = fmaf(u, u, a);
      b = fmaf(W[e], V[e], b);
    }
    const float v = 2.0f * a - b;
    q[c] = v;
    part = v;
  }
  block_add_double(part, dst);
}

__global__ void lincomb_kernel(const float* __restrict__ x, float alpha, const float* __restrict__ y, float beta,
                               float* __restrict__ out, int n) {
  pdl_enter();
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) out[e] = alpha * x[e] + beta * y[e];
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

void k_hutch_data(const float* Lf, const float* Kuu, const float* s, int M, int Mp, const float* Zs, const float* Xs,
                  int D, int B, const float* sf2, const float* m, bool precond, float* bufA, float* bufB,
                  float* bufC, int cmax, float* v, float* colq, double* red, cudaStream_t st) {
  // v = P m~ = 2 T m~ - T K~ T m~ (or m~ without the preconditioner)
  if (precond) {
    tsmm(Lf, Mp, M, true, m, 1, nullptr, bufA, st);          // L^T m
    tsmm(Lf, Mp, M, false, bufA, 1, nullptr, bufB, st);      // T m
    tsmm(Kuu, Mp, M, false, bufB, 1, s, bufA, st);           // K~ T m
    tsmm(Lf, Mp, M, true, bufA, 1, nullptr, bufC, st);       // L^T K~ T m
    tsmm(Lf, Mp, M, false, bufC, 1, nullptr, bufA, st);      // T K~ T m
    svgp_note_launch();
    pdl_launch(lincomb_kernel, (M + 255) / 256, 256, 0, st, bufB, 2.0f, bufA, -1.0f, v, M);
  } else {
    cudaMemcpyAsync(v, m, sizeof(float) * M, cudaMemcpyDeviceToDevice, st);
  }
  // k_n^T P k_n per point, blocks of cmax points
  for (int c0 = 0; c0 < B; c0 += cmax) {
    const int nc = B - c0 < cmax ? B - c0 : cmax;
    const size_t n = (size_t)M * nc;
    svgp_note_launch();
    pdl_launch(kuf_dense_kernel, (int)((n + 255) / 256), 256, 0, st, Zs, Xs, M, D, sf2, c0, nc, bufA);
    tsmm(Lf, Mp, M, true, bufA, nc, nullptr, bufB, st);     // u = L^T Kuf
    tsmm(Lf, Mp, M, false, bufB, nc, nullptr, bufC, st);    // w = L u
    tsmm(Kuu, Mp, M, false, bufC, nc, s, bufA, st);         // K~ w
    svgp_note_launch();
    pdl_launch(colq_kernel, (nc + 127) / 128, 128, 0, st, bufB, bufC, bufA, M, nc, colq + c0, red + RED_PPSI);
  }
}
