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

// y[j] += sum_{i in this block's row range} A[i][j] x[i] (A: Mp x Mp FP32,
// entries beyond M zero): threads over columns (coalesced rows), blocks over
// 256 columns x 512 rows; partial sums by atomics (y zeroed first).
__global__ void __launch_bounds__(256) gemvt_kernel(const float* __restrict__ A, int Mp, int M,
                                                    const float* __restrict__ x, float* __restrict__ y) {
  pdl_enter();
  const int j = blockIdx.x * 256 + threadIdx.x;
  const int i0 = blockIdx.y * 512, i1 = min(M, i0 + 512);
  __shared__ float xs[512];
  for (int e = threadIdx.x; e < 512; e += 256) xs[e] = i0 + e < M ? __ldg(x + i0 + e) : 0.f;
  __syncthreads();
  if (j >= M) return;
  float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
  int i = i0;
  for (; i + 4 <= i1; i += 4) {
    a0 = fmaf(__ldg(A + (size_t)i * Mp + j), xs[i - i0], a0);
    a1 = fmaf(__ldg(A + (size_t)(i + 1) * Mp + j), xs[i + 1 - i0], a1);
    a2 = fmaf(__ldg(A + (size_t)(i + 2) * Mp + j), xs[i + 2 - i0], a2);
    a3 = fmaf(__ldg(A + (size_t)(i + 3) * Mp + j), xs[i + 3 - i0], a3);
  }
  for (; i < i1; ++i) a0 = fmaf(__ldg(A + (size_t)i * Mp + j), xs[i - i0], a0);
  atomicAdd(y + j, (a0 + a1) + (a2 + a3));
}

// out = x + d o y (elementwise, n entries)
__global__ void diagadd_kernel(const float* __restrict__ x, const float* __restrict__ d, const float* __restrict__ y,
                               float* __restrict__ out, int n) {
  pdl_enter();
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) out[e] = fmaf(d[e], y[e], x[e]);
}

__global__ void lincomb_kernel(const float* __restrict__ x, float alpha, const float* __restrict__ y, float beta,
                               float* __restrict__ out, int n) {
  pdl_enter();
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) out[e] = alpha * x[e] + beta * y[e];
}


// ---- tensor-core form: every M x N factor kept as its transpose (N rows of
// Mp, BF16 or hi/lo BF16), the K-major operand of the next product ----
__device__ __forceinline__ float warp_sum32(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}
__device__ __forceinline__ float getv(const bf16* p, size_t i) { return __bfloat162float(p[i]); }
__device__ __forceinline__ float getv(const SplitPtr& p, size_t i) {
  return __bfloat162float(p.hi[i]) + __bfloat162float(p.lo[i]);
}

// K~ = Kuu + diag(s~) (FP32 Kuu, Mp x Mp) in the operand precision.
template <class OutP>
__global__ void kt_op_kernel(const float* __restrict__ Kuu, const float* __restrict__ s, int M, int Mp, OutP out) {
  pdl_enter();
  const int i = blockIdx.y, j = (blockIdx.x * blockDim.x + threadIdx.x) * 4;   // row i, columns j .. j + 3
  if (j >= Mp) return;
  const size_t e = (size_t)i * Mp + j;
  const float4 k = *reinterpret_cast<const float4*>(Kuu + e);
  float v[4] = {k.x, k.y, k.z, k.w};
  if (i < M && i >= j && i < j + 4) v[i - j] += s[i];
  put4(out, e, v);
}

// Rows r < Np of the transposed operand: row r = Kuf column c0 + r (r < nc),
// zero otherwise and beyond column M.
template <class OutP>
__global__ void kuf_t_kernel(const float* __restrict__ Zs, const float* __restrict__ Xs, int M, int Mp, int D,
                             const float* __restrict__ sf2, int c0, int nc, int Np, OutP out) {
  pdl_enter();
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)Np * Mp) return;
  const int r = (int)(e / Mp), i = (int)(e % Mp);
  float v = 0.f;
  if (r < nc && i < M) {
    const int Dp = (D + 3) & ~3;
    const float* z = Zs + (size_t)i * Dp;
    const float* x = Xs + (size_t)(c0 + r) * Dp;
    float d2 = 0.f;
    for (int d = 0; d < D; ++d) {
      const float t = __ldg(z + d) - __ldg(x + d);
      d2 = fmaf(t, t, d2);
    }
    v = *sf2 * expf(-0.5f * d2);
  }
  put(out, e, v);
}

// Rows r < Np: probe column r (r < K; probes M x K row-major), zero otherwise.
template <class OutP>
__global__ void probes_t_kernel(const float* __restrict__ Z, int M, int Mp, int K, int Np, OutP out) {
  pdl_enter();
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)Np * Mp) return;
  const int r = (int)(e / Mp), i = (int)(e % Mp);
  put(out, e, (r < K && i < M) ? Z[(size_t)i * K + r] : 0.f);
}

// q_r = 2 |U_r|^2 - W_r . V_r over the rows r < nc of transposed factors (one
// block of 256 threads per row), into q[r] and, summed, into *dst.
template <class OutP>
__global__ void rowq_kernel(OutP U, OutP W, OutP V, int M, int Mp, int nc, float* __restrict__ q, double* dst) {
  pdl_enter();
  __shared__ float red2[2][8];
  const int r = blockIdx.x, lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  float a = 0.f, b = 0.f;
  for (int i = threadIdx.x; i < M; i += 256) {
    const size_t e = (size_t)r * Mp + i;
    const float u = getv(U, e);
    a = fmaf(u, u, a);
    b = fmaf(getv(W, e), getv(V, e), b);
  }
  a = warp_sum32(a);
  b = warp_sum32(b);
  if (lane == 0) { red2[0][wid] = a; red2[1][wid] = b; }
  __syncthreads();
  double part = 0.0;
  if (threadIdx.x == 0) {
    float sa = 0.f, sb = 0.f;
    for (int w = 0; w < 8; ++w) { sa += red2[0][w]; sb += red2[1][w]; }
    q[r] = 2.0f * sa - sb;
    part = 2.0f * sa - sb;
  }
  block_add_double(part, dst);
}

// *dst += sum over rows r < n and columns i < M of X[r][i] Y[r][i].
template <class XP, class YP>
__global__ void tdot_kernel(XP X, YP Y, int M, int Mp, int n, double* dst) {
  pdl_enter();
  double part = 0.0;
  const size_t tot = (size_t)n * Mp;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x)
    if ((int)(e % Mp) < M) part += (double)getv(X, e) * (double)getv(Y, e);
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

void gemvt(const float* A, int Mp, int M, const float* x, float* y, cudaStream_t st) {
  k_zero(st, y, sizeof(float) * (size_t)M);
  svgp_note_launch();
  pdl_launch(gemvt_kernel, dim3((M + 255) / 256, (M + 511) / 512), 256, 0, st, A, Mp, M, x, y);
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
  // v = P m~ = 2 T m~ - T K~ T m~ (or m~ without the preconditioner), by
  // matrix-vector products (the FP32 GEMV for L x and Kuu x)
  if (precond) {
    gemvt(Lf, Mp, M, m, bufA, st);                                                  // L^T m
    k_gemv(Lf, Mp, M, bufA, 1.f, nullptr, 0.f, bufB, nullptr, nullptr, st);       // T m
    k_gemv(Kuu, Mp, M, bufB, 1.f, nullptr, 0.f, bufC, nullptr, nullptr, st);      // Kuu T m
    svgp_note_launch();
    pdl_launch(diagadd_kernel, (M + 255) / 256, 256, 0, st, bufC, s, bufB, bufA, M);   // K~ T m
    gemvt(Lf, Mp, M, bufA, bufC, st);                                               // L^T K~ T m
    k_gemv(Lf, Mp, M, bufC, 1.f, nullptr, 0.f, bufA, nullptr, nullptr, st);       // T K~ T m
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

template <class OutP>
void k_kt_op(const float* Kuu, const float* s, int M, int Mp, OutP out, cudaStream_t st) {
  svgp_note_launch();
  pdl_launch(kt_op_kernel<OutP>, dim3((Mp / 4 + 127) / 128, Mp), 128, 0, st, Kuu, s, M, Mp, out);
}
template <class OutP>
void k_kuf_t(const float* Zs, const float* Xs, int M, int Mp, int D, const float* sf2, int c0, int nc, int Np,
             OutP out, cudaStream_t st) {
  svgp_note_launch();
  pdl_launch(kuf_t_kernel<OutP>, (int)(((size_t)Np * Mp + 255) / 256), 256, 0, st, Zs, Xs, M, Mp, D, sf2, c0, nc,
             Np, out);
}
template <class OutP>
void k_probes_t(const float* Z, int M, int Mp, int K, int Np, OutP out, cudaStream_t st) {
  svgp_note_launch();
  pdl_launch(probes_t_kernel<OutP>, (int)(((size_t)Np * Mp + 255) / 256), 256, 0, st, Z, M, Mp, K, Np, out);
}
template <class OutP>
void k_rowq(OutP U, OutP W, OutP V, int M, int Mp, int nc, float* q, double* dst, cudaStream_t st) {
  svgp_note_launch();
  pdl_launch(rowq_kernel<OutP>, nc, 256, 0, st, U, W, V, M, Mp, nc, q, dst);
}
template <class OutP>
void k_tdot(OutP X, OutP Y, int M, int Mp, int n, double* dst, cudaStream_t st) {
  size_t tot = (size_t)n * Mp;
  int grid = (int)((tot + 255) / 256);
  if (grid > 1024) grid = 1024;
  svgp_note_launch();
  pdl_launch(tdot_kernel<OutP, OutP>, grid, 256, 0, st, X, Y, M, Mp, n, dst);
}
#define SVGP_HT_INST(T)                                                                                      \
  template void k_kt_op<T>(const float*, const float*, int, int, T, cudaStream_t);                          \
  template void k_kuf_t<T>(const float*, const float*, int, int, int, const float*, int, int, int, T,        \
                           cudaStream_t);                                                                     \
  template void k_probes_t<T>(const float*, int, int, int, int, T, cudaStream_t);                            \
  template void k_rowq<T>(T, T, T, int, int, int, float*, double*, cudaStream_t);                            \
  template void k_tdot<T>(T, T, int, int, int, double*, cudaStream_t);
SVGP_HT_INST(bf16*)
SVGP_HT_INST(SplitPtr)
