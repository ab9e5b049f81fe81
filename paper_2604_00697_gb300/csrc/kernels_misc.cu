// Elementwise, GEMV and reduction kernels of the R-SVGP step: SE-ARD blocks,
// factor preparation, predictive means, Gaussian per-point terms, gradient
// assembly, FP64 scalar finalisation and the fused Adam update.
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace {

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// z~ = z / ell, x~ = x / ell, padded to Dp = round_up(D, 4) columns and (for
// Z) Mp rows, padding zero.
__global__ void prep_coords_kernel(const float* __restrict__ Z, const float* __restrict__ X,
                                   const float* __restrict__ ell, int M, int Mp, int B, int D,
                                   float* __restrict__ Zs, float* __restrict__ Xs, const float* __restrict__ s,
                                   double* logs) {
  pdl_enter();
  int Dp = (D + 3) & ~3;
  int tot = (Mp + B) * Dp;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += gridDim.x * blockDim.x) {
    int r = e / Dp, d = e % Dp;
    if (r < Mp) {
      Zs[e] = (r < M && d < D) ? Z[(size_t)r * D + d] / ell[d] : 0.f;
    } else {
      int n = r - Mp;
      Xs[(size_t)n * Dp + d] = (d < D) ? X[(size_t)n * D + d] / ell[d] : 0.f;
    }
  }
  // *logs += sum_i log s~_i (the log-det of diag(s~) in the KL term), by the
  // blocks whose first index is below M
  if (logs && blockIdx.x * blockDim.x < M) {
    double part = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) part += log((double)s[i]);
    block_add_double(part, logs);
  }
}

// Kuu = sf2 exp(-1/2 ||z~_i - z~_j||^2) (per-dimension differences), exact
// sf2 on the diagonal, zero padding.  64 x 64 tiles (16 elements per thread),
// points staged in shared memory.  Only the tiles on and below the diagonal
// are computed (blockIdx.x enumerates them row by row); an off-diagonal tile
// is also written transposed, through shared memory -- (a - b)^2 = (b - a)^2
// exactly, so the mirror is the value the upper tile would compute.
template <class OutP, int DP>
__global__ void __launch_bounds__(256) kuu_kernel(const float* __restrict__ Zs, int M, int Mp, int D,
                                                  const float* __restrict__ sf2p, float* __restrict__ Kf,
                                                  OutP Klo, bool has_lo) {
  pdl_enter();
  __shared__ float zi[64][DP + 1], zj[64][DP + 1];
  __shared__ float tile[64][65];
  const int Dp = (D + 3) & ~3;
  // lower-triangle tile t -> (bi, bj), bj <= bi
  const int t = blockIdx.x;
  int bi = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
  while ((bi + 1) * (bi + 2) / 2 <= t) ++bi;
  while (bi * (bi + 1) / 2 > t) --bi;
  const int bj = t - bi * (bi + 1) / 2;
  const int i0 = bi * 64, j0 = bj * 64;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int e = ty * 32 + tx; e < 64 * DP; e += 256) {
    const int r = e / DP, d = e % DP;
    zi[r][d] = d < Dp ? Zs[(size_t)(i0 + r) * Dp + d] : 0.f;
    zj[r][d] = d < Dp ? Zs[(size_t)(j0 + r) * Dp + d] : 0.f;
  }
  __syncthreads();
  const float sf2 = *sf2p;
  // this thread's two columns z~_j in registers; z~_i read as warp broadcasts
  float zc[2][DP];
#pragma unroll
  for (int cj = 0; cj < 2; ++cj)
#pragma unroll
    for (int d = 0; d < DP; ++d) zc[cj][d] = zj[tx + 32 * cj][d];
#pragma unroll 2
  for (int ri = 0; ri < 8; ++ri) {
    const int rr = ty + 8 * ri, i = i0 + rr;
    float r2[2] = {0.f, 0.f};
#pragma unroll
    for (int d = 0; d < DP; ++d) {
      const float a = zi[rr][d];
#pragma unroll
      for (int cj = 0; cj < 2; ++cj) { const float e = a - zc[cj][d]; r2[cj] = fmaf(e, e, r2[cj]); }
    }
    float val[2];
#pragma unroll
    for (int cj = 0; cj < 2; ++cj) {
      const int j = j0 + tx + 32 * cj;
      float v = (i == j) ? sf2 : sf2 * expf(-0.5f * r2[cj]);
      val[cj] = (i < M && j < M) ? v : 0.f;
    }
#pragma unroll
    for (int cj = 0; cj < 2; ++cj) {
      const size_t o = (size_t)i * Mp + j0 + tx + 32 * cj;
      Kf[o] = val[cj];
      if (has_lo) put(Klo, o, val[cj]);
      tile[rr][tx + 32 * cj] = val[cj];
    }
  }
  if (bi == bj) return;
  __syncthreads();
  // mirror: Kuu[j0 + r][i0 + c] = tile[c][r]
#pragma unroll 2
  for (int r = ty; r < 64; r += 8) {
#pragma unroll
    for (int cj = 0; cj < 2; ++cj) {
      const int c = tx + 32 * cj;
      const size_t o = (size_t)(j0 + r) * Mp + i0 + c;
      const float v = tile[c][r];
      Kf[o] = v;
      if (has_lo) put(Klo, o, v);
    }
  }
}

// L (M x M, ld M, lower) -> Lf (Mp x Mp FP32), Llo, Ltlo = Llo^T (operand
// precision); strictly-upper entries forced to zero; sum log|L_ii|.
template <class OutP>
__global__ void prep_L_kernel(const float* __restrict__ Lin, int M, int Mp, float* __restrict__ Lf,
                              OutP Llo, OutP Ltlo, double* logdet) {
  pdl_enter();
  // block: a strip of 128 rows x 32 columns (sixteen rows per thread)
  __shared__ float tile[128][33];
  const int i0 = blockIdx.y * 128, j0 = blockIdx.x * 32;
  // Strips strictly above the diagonal stay zero in L (and below it in L^T):
  // nothing else ever writes there, and the buffers start zeroed.
  if (j0 > i0 + 127) return;
  const int tx = threadIdx.x;
  double ld = 0.0;
#pragma unroll 4
  for (int ty = threadIdx.y; ty < 128; ty += blockDim.y) {
    const int i = i0 + ty, j = j0 + tx;
    const float val = (i < M && j < M && j <= i) ? Lin[(size_t)i * M + j] : 0.f;
    Lf[(size_t)i * Mp + j] = val;
    put(Llo, (size_t)i * Mp + j, val);
    tile[ty][tx] = val;
    if (i == j && i < M) ld += (double)logf(fabsf(val));
  }
  __syncthreads();
#pragma unroll 4
  for (int e = threadIdx.y; e < 4 * 32; e += blockDim.y) {
    // Lt[j0 + r][i0 + 32 c + tx] = L[i0 + 32 c + tx][j0 + r]
    const int r = e & 31, c = e >> 5;
    put(Ltlo, (size_t)(j0 + r) * Mp + i0 + 32 * c + tx, tile[32 * c + tx][r]);
  }
  if (logdet && j0 >= i0) block_add_double(ld, logdet);
}

// y = alpha * A (x + beta * x2)  (A: Mp x Mp FP32, rows < M); one warp per
// row.  A lane issues the loads of its first 16 float4 of the row before the
// combined vector is staged in shared memory (Mp floats of dynamic shared
// memory), so the row's memory latency overlaps the staging; longer rows
// continue in chunks of 16 float4 per lane.  Optionally
// dot_out += sum_i y_i dotw_i.
__global__ void __launch_bounds__(256) gemv_kernel(const float* __restrict__ A, int Mp, int M,
                                                   const float* __restrict__ x, float alpha,
                                                   const float* __restrict__ x2, float beta, float* __restrict__ y,
                                                   const float* __restrict__ dotw, double* dot_out) {
  pdl_enter();
  extern __shared__ float xs[];
  constexpr int CH = 16;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int n4 = Mp / 4;
  const bool live = warp < M;
  const float4* row = reinterpret_cast<const float4*>(A + (size_t)(live ? warp : 0) * Mp);
  float4 a[CH];
#pragma unroll
  for (int u = 0; u < CH; ++u) {
    const int k = lane + 32 * u;
    a[u] = (live && k < n4) ? __ldg(row + k) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  // staging: eight loads in flight per thread before the shared-memory stores
  for (int j0 = threadIdx.x; j0 < Mp; j0 += 8 * blockDim.x) {
    float xv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int j = j0 + u * blockDim.x;
      xv[u] = j < M ? __ldg(x + j) : 0.f;
      if (x2 && j < M) xv[u] = fmaf(beta, __ldg(x2 + j), xv[u]);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int j = j0 + u * blockDim.x;
      if (j < Mp) xs[j] = xv[u];
    }
  }
  __syncthreads();
  double part = 0.0;
  if (live) {
    const float4* xv = reinterpret_cast<const float4*>(xs);
    float acc0 = 0.f, acc1 = 0.f;
    for (int k0 = 0;; k0 += 32 * CH) {
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        const int k = min(k0 + lane + 32 * u, n4 - 1);
        const float4 b = xv[k];
        acc0 = fmaf(a[u].x, b.x, acc0); acc1 = fmaf(a[u].y, b.y, acc1);
        acc0 = fmaf(a[u].z, b.z, acc0); acc1 = fmaf(a[u].w, b.w, acc1);
      }
      if (k0 + 32 * CH >= n4) break;
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        const int k = k0 + 32 * CH + lane + 32 * u;
        a[u] = k < n4 ? __ldg(row + k) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    const float acc = warp_sum(acc0 + acc1) * alpha;
    if (lane == 0) {
      y[warp] = acc;
      if (dotw) part = (double)acc * dotw[warp];
    }
  }
  if (dot_out) block_add_double(part, dot_out);
}

constexpr float HALF_LOG2E = 0.72134752044448170f;   // log2(e) / 2

__device__ __forceinline__ float ex2f(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Calls KERNEL<DP> with DP the smallest of 4, 8, 16, 32 not below D.
#define SVGP_DP_DISPATCH(D, ...)                              \
  do {                                                        \
    if ((D) <= 4) { constexpr int DP = 4; __VA_ARGS__; }      \
    else if ((D) <= 8) { constexpr int DP = 8; __VA_ARGS__; } \
    else if ((D) <= 16) { constexpr int DP = 16; __VA_ARGS__; } \
    else { constexpr int DP = 32; __VA_ARGS__; }              \
  } while (0)

// mu_n += sum_{i in chunk} Kuf_in v_i.  grid (ceil(B/512), ceil(M/64)).
template <int DP>
__global__ void mu_kernel(const float* __restrict__ Zs, const float* __restrict__ Xs, int M, int B,
                          int D, const float* __restrict__ sf2p, const float* __restrict__ v,
                          float* __restrict__ mu) {
  pdl_enter();
  __shared__ float zs[64][DP + 1];
  __shared__ float vs[64];
  const int Dp = (D + 3) & ~3;
  int i0 = blockIdx.y * 64;
  int ni = min(64, M - i0);
  for (int e = threadIdx.x; e < 64 * DP; e += blockDim.x) {
    int r = e / DP, d = e % DP;
    zs[r][d] = (r < ni && d < Dp) ? Zs[(size_t)(i0 + r) * Dp + d] : 0.f;
  }
  for (int r = threadIdx.x; r < 64; r += blockDim.x) vs[r] = r < ni ? v[i0 + r] : 0.f;
  __syncthreads();
  // four points per thread: each shared-memory z~_i row feeds four distances
  constexpr int NP = 4;
  const int nb = blockIdx.x * blockDim.x * NP + threadIdx.x;
  float x[NP][DP];
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const int n = nb + p * blockDim.x;
#pragma unroll
    for (int d = 0; d < DP; ++d) x[p][d] = (n < B && d < Dp) ? Xs[(size_t)n * Dp + d] : 0.f;
  }
  const float l2sf2 = log2f(*sf2p);
  float acc[NP] = {0.f, 0.f, 0.f, 0.f};
  for (int r = 0; r < ni; ++r) {
    float r2[NP] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int d = 0; d < DP; ++d) {
      const float zd = zs[r][d];
#pragma unroll
      for (int p = 0; p < NP; ++p) { const float e = zd - x[p][d]; r2[p] = fmaf(e, e, r2[p]); }
    }
    const float vr = vs[r];
#pragma unroll
    for (int p = 0; p < NP; ++p) acc[p] = fmaf(ex2f(fmaf(-HALF_LOG2E, r2[p], l2sf2)), vr, acc[p]);
  }
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const int n = nb + p * blockDim.x;
    if (n < B) atomicAdd(mu + n, acc[p]);
  }
}

__global__ void pointwise_gauss_kernel(const float* __restrict__ y, const float* __restrict__ mu,
                                       const float* __restrict__ noise, int B, float* __restrict__ g,
                                       double* red) {
  pdl_enter();
  double part = 0.0;
  float inv = 1.0f / *noise;
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < B; n += gridDim.x * blockDim.x) {
    float r = y[n] - mu[n];
    if (g) g[n] = r * inv;
    part += (double)r * r;
  }
  block_add_double(part, red + RED_SQERR);
}

// Kg_i += sum_{n in chunk} Kuf_in g_n.  grid (ceil(M/512), ceil(B/64)).
template <int DP>
__global__ void kg_kernel(const float* __restrict__ Zs, const float* __restrict__ Xs, int M, int B,
                          int D, const float* __restrict__ sf2p, const float* __restrict__ g,
                          float* __restrict__ Kg) {
  pdl_enter();
  __shared__ float xs[64][DP + 1];
  __shared__ float gs[64];
  const int Dp = (D + 3) & ~3;
  int n0 = blockIdx.y * 64;
  int nn = min(64, B - n0);
  for (int e = threadIdx.x; e < 64 * DP; e += blockDim.x) {
    int r = e / DP, d = e % DP;
    xs[r][d] = (r < nn && d < Dp) ? Xs[(size_t)(n0 + r) * Dp + d] : 0.f;
  }
  for (int r = threadIdx.x; r < 64; r += blockDim.x) gs[r] = r < nn ? g[n0 + r] : 0.f;
  __syncthreads();
  // four inducing points per thread
  constexpr int NP = 4;
  const int ib = blockIdx.x * blockDim.x * NP + threadIdx.x;
  float z[NP][DP];
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const int i = ib + p * blockDim.x;
#pragma unroll
    for (int d = 0; d < DP; ++d) z[p][d] = (i < M && d < Dp) ? Zs[(size_t)i * Dp + d] : 0.f;
  }
  const float l2sf2 = log2f(*sf2p);
  float acc[NP] = {0.f, 0.f, 0.f, 0.f};
  for (int r = 0; r < nn; ++r) {
    float r2[NP] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int d = 0; d < DP; ++d) {
      const float xd = xs[r][d];
#pragma unroll
      for (int p = 0; p < NP; ++p) { const float e = xd - z[p][d]; r2[p] = fmaf(e, e, r2[p]); }
    }
    const float gr = gs[r];
#pragma unroll
    for (int p = 0; p < NP; ++p) acc[p] = fmaf(ex2f(fmaf(-HALF_LOG2E, r2[p], l2sf2)), gr, acc[p]);
  }
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const int i = ib + p * blockDim.x;
    if (i < M) atomicAdd(Kg + i, acc[p]);
  }
}

// Symmetrised G_P = c/2 (Kg m^T + m Kg^T) + c/(2 noise) Psi + Kuu/2
//                   - (m w^T + w m^T)/2, zero padding.
template <class OutP>
__global__ void gp_assemble_kernel(const float* __restrict__ Kuu, const float* __restrict__ Psi,
                                   const float* __restrict__ Kg, const float* __restrict__ m,
                                   const float* __restrict__ w, const float* __restrict__ noise, float c,
                                   int M, int Mp, OutP out) {
  pdl_enter();
  // block: row i = blockIdx.y, 4 consecutive columns per thread
  const float cn = noise ? c * 0.5f / *noise : c;   // probit: Psi = Kuf diag(|h|) Kuf^T
  const int i = blockIdx.y;
  const int j = (blockIdx.x * blockDim.x + threadIdx.x) * 4;
  if (j >= Mp) return;
  const size_t e = (size_t)i * Mp + j;
  const float4 ps = __ldg(reinterpret_cast<const float4*>(Psi + e));
  const float4 ku = __ldg(reinterpret_cast<const float4*>(Kuu + e));
  const float pv[4] = {ps.x, ps.y, ps.z, ps.w}, kv[4] = {ku.x, ku.y, ku.z, ku.w};
  const bool row_ok = i < M;
  const bool mt = m != nullptr;   // the m~ terms of the preconditioned bound
  const float kgi = row_ok ? Kg[i] : 0.f, mi = (row_ok && mt) ? m[i] : 0.f, wi = row_ok ? w[i] : 0.f;
  // Kg and w are Mp-long workspace vectors (16-byte aligned): one vector load
  // each; m~ is the caller's (any alignment, M long): scalar loads
  float kgv[4] = {0.f, 0.f, 0.f, 0.f}, wv[4] = {0.f, 0.f, 0.f, 0.f}, mv[4] = {0.f, 0.f, 0.f, 0.f};
  if (mt && row_ok) {
    const float4 k4 = __ldg(reinterpret_cast<const float4*>(Kg + j));
    const float4 w4 = __ldg(reinterpret_cast<const float4*>(w + j));
    kgv[0] = k4.x; kgv[1] = k4.y; kgv[2] = k4.z; kgv[3] = k4.w;
    wv[0] = w4.x; wv[1] = w4.y; wv[2] = w4.z; wv[3] = w4.w;
#pragma unroll
    for (int q = 0; q < 4; ++q) mv[q] = j + q < M ? __ldg(m + j + q) : 0.f;
  }
  float val[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int jj = j + q;
    val[q] = 0.f;
    if (row_ok && jj < M) {
      val[q] = cn * pv[q] + 0.5f * kv[q];
      if (mt) val[q] += 0.5f * c * (kgi * mv[q] + mi * kgv[q]) - 0.5f * (mi * wv[q] + wi * mv[q]);
    }
  }
  put4(out, e, val);
}

// Kuu-side chain rule: with A_ij = G_Kuu_ij Kuu_ij and e_d = z~_jd - z~_id,
//   rowacc[i][d] += sum_j A_ij e_d,  rowacc[i][D + d] += sum_j A_ij e_d^2,
//   rowacc[i][2D] += sum_j A_ij.
// Accumulated in the expanded form S0 = sum_j A_ij, S1_d = sum_j A_ij z~_jd,
// S2_d = sum_j A_ij z~_jd^2 (two FMAs per dimension and element) and reported
// as S1_d - z~_id S0 and S2_d - 2 z~_id S1_d + z~_id^2 S0.
// Block = 32 rows (lane = row i) x a range of JB columns j, split over the 8
// warps; the host sizes JB so that the grid fills the SMs in one wave.  A is
// symmetric, so A_ij is read as A[j][i]: a warp reads 32 consecutive floats of
// row j (eight rows in flight per warp).  z~_j of the range is staged in
// shared memory; the broadcast reads of it bound the loop, so groups of four
// lanes share them: lane r of a group accumulates S1, S2 of the group's four
// rows for its quarter of the dimensions (DQ of them), taking the other rows'
// A_ij by shuffles, and reads only its DQ values of z~_j.
// Warp partials meet in shared memory; one atomic per row and value per block.
template <int DP>
constexpr int kuu_zw() { return 4 * ((DP / 4 + 1) & ~1); }   // staged floats per z~ row (4 lane slots)

template <int DP>
__global__ void __launch_bounds__(256) kuu_bwd_kernel(const float* __restrict__ GK, const float* __restrict__ Kuu,
                                                     const float* __restrict__ Zs, int M, int Mp, int D,
                                                     float* __restrict__ rowacc, int JB) {
  pdl_enter();
  constexpr int U = 8;
  constexpr int DQ = DP / 4, DQP = (DQ + 1) & ~1, ZW = kuu_zw<DP>();
  extern __shared__ __align__(16) float zs[];      // [JB][ZW]: lane slot r holds dimensions r DQ .. + DQ
  __shared__ float part[32][2 * DP + 2];           // raw sums per row: S1 [0, D), S2 [D, 2D), S0 2D
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, r4 = lane & 3;
  const int i = blockIdx.x * 32 + lane;
  const int Dp = (D + 3) & ~3;
  const int jb = blockIdx.y * JB, je = min(M, jb + JB);
  for (int e = threadIdx.x; e < 32 * (2 * DP + 2); e += 256) (&part[0][0])[e] = 0.f;
#pragma unroll 8
  for (int e = threadIdx.x; e < JB * ZW; e += 256) {
    const int r = e / ZW, sl = e - r * ZW, jj = sl % DQP, d = (sl / DQP) * DQ + jj;
    zs[e] = (jb + r < je && jj < DQ && d < Dp) ? __ldg(Zs + (size_t)(jb + r) * Dp + d) : 0.f;
  }
  // S1p[k][q] = (S1, S1) of row 4 (lane / 4) + (r4 ^ k) at dimensions r4 DQ + 2q, 2q + 1
  f32x2 S1p[4][DQP / 2], S2p[4][DQP / 2];
  float S0 = 0.f;
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int q = 0; q < DQP / 2; ++q) { S1p[k][q] = 0ull; S2p[k][q] = 0ull; }
  __syncthreads();
  const bool row_ok = i < M;
  for (int j = jb + warp; j < je; j += 8 * U) {
    float a[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int jj = j + 8 * u;
      a[u] = (row_ok && jj < je) ? __ldg(GK + (size_t)jj * Mp + i) * __ldg(Kuu + (size_t)jj * Mp + i) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int jj = min(j + 8 * u, je - 1) - jb;
      const float* zr = &zs[jj * ZW + r4 * DQP];
      f32x2 zp[DQP / 2], zq[DQP / 2];
      if (DQP % 4 == 0) {
#pragma unroll
        for (int q = 0; q < DQP / 4; ++q) {
          const ulonglong2 v = reinterpret_cast<const ulonglong2*>(zr)[q];
          zp[2 * q] = v.x;
          zp[2 * q + 1] = v.y;
        }
      } else {
#pragma unroll
        for (int q = 0; q < DQP / 2; ++q) zp[q] = reinterpret_cast<const f32x2*>(zr)[q];
      }
#pragma unroll
      for (int q = 0; q < DQP / 2; ++q) zq[q] = mul2(zp[q], zp[q]);
      S0 += a[u];
      float ak[4];
      ak[0] = a[u];
      ak[1] = __shfl_xor_sync(0xffffffffu, a[u], 1);
      ak[2] = __shfl_xor_sync(0xffffffffu, a[u], 2);
      ak[3] = __shfl_xor_sync(0xffffffffu, a[u], 3);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const f32x2 a2 = pack2(ak[k], ak[k]);
#pragma unroll
        for (int q = 0; q < DQP / 2; ++q) {
          fma2(S1p[k][q], a2, zp[q]);
          fma2(S2p[k][q], a2, zq[q]);
        }
      }
    }
  }
  // raw sums of the eight warps into part
  atomicAdd(&part[lane][2 * D], S0);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int rr = (lane & ~3) + (r4 ^ k);
#pragma unroll
    for (int q = 0; q < DQP / 2; ++q) {
      float s1a, s1b, s2a, s2b;
      unpack2(S1p[k][q], s1a, s1b);
      unpack2(S2p[k][q], s2a, s2b);
      const int d0 = r4 * DQ + 2 * q;
      if (2 * q < DQ && d0 < D) {
        atomicAdd(&part[rr][d0], s1a);
        atomicAdd(&part[rr][D + d0], s2a);
      }
      if (2 * q + 1 < DQ && d0 + 1 < D) {
        atomicAdd(&part[rr][d0 + 1], s1b);
        atomicAdd(&part[rr][D + d0 + 1], s2b);
      }
    }
  }
  __syncthreads();
  // difference form per row, one global atomic per row and value
  const int Wd = 2 * D + 1;
  for (int e = threadIdx.x; e < 32 * Wd; e += 256) {
    const int r = e / Wd, k = e - r * Wd;
    const int ii = blockIdx.x * 32 + r;
    if (ii >= M) continue;
    const float s0 = part[r][2 * D];
    float v = s0;
    if (k < D) {
      v = fmaf(-__ldg(Zs + (size_t)ii * Dp + k), s0, part[r][k]);
    } else if (k < 2 * D) {
      const int d = k - D;
      const float z = __ldg(Zs + (size_t)ii * Dp + d);
      v = fmaf(z, fmaf(z, s0, -2.0f * part[r][d]), part[r][k]);
    }
    atomicAdd(rowacc + (size_t)ii * Wd + k, v);
  }
}

__global__ void logs_kernel(const float* __restrict__ s, int M, double* red) {
  pdl_enter();
  double part = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x)
    part += log((double)s[i]);
  block_add_double(part, red + RED_LOGS);
}

// dZ_id = (rowacc_f[i][d] + 2 rowacc_u[i][d]) / ell_d for a block of RB = 8 rows;
// then the column sums of the lengthscale parts rowacc_f[i][D + d] +
// rowacc_u[i][D + d] and of the signal-variance parts rowacc_*[i][2D] over the
// block's rows (FP32), added in FP64 to acc_ell and the reduction slots (one
// atomic per block and value).  With nparts > 0 the data part rowacc_f is the
// sum of nparts partial row sets rowpart[p][k][i] (k < 2D + 1, i < Mp), added
// here in a fixed order.
__global__ void __launch_bounds__(256) grad_finalize_kernel(const float* __restrict__ rf, const float* __restrict__ ru,
                                                            const float* __restrict__ rowpart, int nparts, int Mp,
                                                            const float* __restrict__ ell, int M, int D,
                                                            float* __restrict__ dZ, double* acc_ell, double* red) {
  pdl_enter();
  constexpr int RB = 8;
  __shared__ float tf[RB][2 * SVGP_MAXD + 2], tu[RB][2 * SVGP_MAXD + 2];
  const int W = 2 * D + 1;
  const int r0 = blockIdx.x * RB;
  const int nr = min(RB, M - r0);
  for (int e = threadIdx.x; e < RB * W; e += blockDim.x) {
    const int k = e / RB, r = e - k * RB;
    float v = 0.f;
    if (r < nr) {
      if (nparts > 0) {
        const float* pp = rowpart + (size_t)k * Mp + r0 + r;
        const size_t stride = (size_t)W * Mp;
        // eight loads in flight, added in part order
        int p = 0;
        for (; p + 8 <= nparts; p += 8) {
          float a[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) a[u] = __ldg(pp + (p + u) * stride);
#pragma unroll
          for (int u = 0; u < 8; ++u) v += a[u];
        }
        float a[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) a[u] = p + u < nparts ? __ldg(pp + (p + u) * stride) : 0.f;
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (p + u < nparts) v += a[u];
      } else {
        v = rf[(size_t)(r0 + r) * W + k];
      }
    }
    tf[r][k] = v;
    tu[r][k] = r < nr ? ru[(size_t)(r0 + r) * W + k] : 0.f;     // staged: the sums below read it per row
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nr * D; e += blockDim.x) {
    const int r = e / D, d = e - r * D;
    dZ[(size_t)r0 * D + e] = (tf[r][d] + 2.0f * tu[r][d]) / ell[d];
  }
  // column sums: thread t < D -> lengthscale d = t; t == D -> data part of the
  // signal variance; t == D + 1 -> Kuu part
  const int t = threadIdx.x;
  if (t < D + 2) {
    float acc = 0.f;
    for (int r = 0; r < nr; ++r) {
      if (t < D) acc += tf[r][D + t] + tu[r][D + t];
      else if (t == D) acc += tf[r][2 * D];
      else acc += tu[r][2 * D];
    }
    if (t < D) atomicAdd(acc_ell + t, (double)acc);
    else if (t == D) atomicAdd(red + RED_SUMA_F, (double)acc);
    else atomicAdd(red + RED_SUMA_U, (double)acc);
  }
}

// Scalar assembly of Eq. (7) in FP64 (and the scalar gradients).  FP64
// divisions and logarithms are long dependent chains on this part, so the
// independent results go to different warps: warp 0 lane d the lengthscale
// gradient d, warp 1 the bound's terms, warp 2 the sf2 and noise gradients.
__global__ void terms_finalize_kernel(const double* __restrict__ red, const double* __restrict__ acc_ell,
                                      const float* __restrict__ sf2p, const float* __restrict__ noisep,
                                      const float* __restrict__ ell, int M, int D, int B, double N, bool probit,
                                      int hutch_K, double* terms, float* dsf2, float* dnoise, float* dell,
                                      int* errword) {
  pdl_enter();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    if (dsf2 && lane < D) dell[lane] = (float)(acc_ell[lane] / ell[lane]);
    return;
  }
  if (lane != 0) return;
  const double noise = probit ? 1.0 : *noisep, c = N / B;
  const double sqerr = probit ? 0.0 : red[RED_SQERR];
  if (warp == 2) {
    if (dsf2) {
      const double sf2 = *sf2p;
      // sum_n sigma_n^2 as below
      const double sumvar = probit ? red[RED_SUMVAR] : (double)B * sf2 - red[RED_PPSI];
      const double sumh = probit ? red[RED_SUMH] : -0.5 * B / noise;   // sum_n h_n
      *dsf2 = (float)(c * sumh + (red[RED_SUMA_F] + red[RED_SUMA_U]) / sf2);
      *dnoise = probit ? 0.f : (float)(c * (-0.5 * B / noise + (sqerr + sumvar) / (2.0 * noise * noise)));
    }
    return;
  }
  const double sf2 = *sf2p;
  double trA1 = red[RED_TRA1], froA1 = red[RED_FROA1];
  double trPKt = 2.0 * trA1 - froA1;                 // tr(P K~) = tr((2I - A1) A1)
  double trPKuu = trPKt - red[RED_SPDIAG];            // minus tr(P diag(s))
  if (hutch_K > 0) {                                  // Section 3.4 estimates
    trA1 = red[RED_HKT] / hutch_K;
    trPKuu = (2.0 * red[RED_HW1] - red[RED_HX4]) / hutch_K;
  }
  double quad = red[RED_QUAD];
  double logdetT = 2.0 * red[RED_LOGDETL];
  double logdetS = red[RED_LOGS];
  // sum_n sigma_n^2: Gaussian from sum_n sf2 - k_n^T P k_n = B sf2 - <P, Psi>; probit per point
  double sumvar = probit ? red[RED_SUMVAR] : (double)B * sf2 - red[RED_PPSI];
  const double LOG2PI = 1.8378770664093453;
  double E = probit ? c * red[RED_ELL]
                    : c * (-0.5 * B * (LOG2PI + log(noise)) - (sqerr + sumvar) / (2.0 * noise));
  double KL = 0.5 * (-trPKuu + trA1 - M + quad - logdetT - logdetS);
  double F = E - KL;
  if (terms) {
    terms[SVGP_T_F] = F; terms[SVGP_T_E] = E; terms[SVGP_T_KL] = KL; terms[SVGP_T_TRKT] = trA1;
    terms[SVGP_T_TRPKUU] = trPKuu; terms[SVGP_T_QUAD] = quad; terms[SVGP_T_LOGDETT] = logdetT;
    terms[SVGP_T_SQERR] = sqerr; terms[SVGP_T_SUMVAR] = sumvar; terms[SVGP_T_LOGDETS] = logdetS;
    terms[SVGP_T_NCLAMP] = probit ? red[RED_NCLAMP] : 0.0;
  }
  if (!isfinite(F)) atomicOr(errword, ERRBIT_NONFINITE);
}

__global__ void predict_finalize_kernel(const float* __restrict__ colsum, const float* __restrict__ sf2,
                                        const float* __restrict__ noise, int Ns, int inc,
                                        float* __restrict__ var) {
  pdl_enter();
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= Ns) return;
  float v = *sf2 - colsum[n];
  if (inc) v += *noise;
  var[n] = v;
}

__device__ __forceinline__ float softplus_f(float x) { return x > 20.f ? x : log1pf(expf(x)); }
__device__ __forceinline__ float sigmoid_f(float x) { return 1.0f / (1.0f + expf(-x)); }

// Adam ascent on the flat vector [Z | ell | sf2 | noise | m | s].
__global__ void adam_kernel(float* __restrict__ raw, float* __restrict__ cons, const float* __restrict__ grad,
                            float* __restrict__ m1, float* __restrict__ m2, const int* __restrict__ step,
                            const float* __restrict__ hyper, const float* __restrict__ zbeta1, int M, int D) {
  pdl_enter();
  int n = M * D + D + 2 + 2 * M;
  int t = *step + 1;
  float lr = hyper[0], b1 = hyper[1], b2 = hyper[2], eps = hyper[3];
  float b1z = zbeta1 ? *zbeta1 : b1;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    int blk;
    if (e < M * D) blk = 0;
    else if (e < M * D + D) blk = 1;
    else if (e == M * D + D) blk = 2;
    else if (e == M * D + D + 1) blk = 3;
    else if (e < M * D + D + 2 + M) blk = 4;
    else blk = 5;
    bool pos = (blk == 1 || blk == 2 || blk == 3 || blk == 5);
    float x = raw[e];
    float g = grad[e];
    if (pos) g *= sigmoid_f(x);
    float bb1 = blk == 0 ? b1z : b1;
    float mm = bb1 * m1[e] + (1.f - bb1) * g;
    float vv = b2 * m2[e] + (1.f - b2) * g * g;
    m1[e] = mm;
    m2[e] = vv;
    float mh = mm / (1.f - powf(bb1, (float)t));
    float vh = vv / (1.f - powf(b2, (float)t));
    x += lr * hyper[4 + blk] * mh / (sqrtf(vh) + eps);
    raw[e] = x;
    cons[e] = pos ? softplus_f(x) : x;
  }
}

__global__ void step_inc_kernel(int* step) {
  pdl_enter(); if (threadIdx.x == 0 && blockIdx.x == 0) *step += 1; }

// Eq. (8) residual of the current iterate; stops the loop (done = 1) when it
// is below eps, or when it is not finite (a diverging step size or a
// non-finite L or K~), which also sets the device error word.
__global__ void ng_check_kernel(double* red, int M, double eps, int* done, int* iters,
                                double* resid, int* errword) {
  pdl_enter();
  if (threadIdx.x != 0) return;
  if (*done) return;
  double r = sqrt(red[RED_NG_RESID] / M);
  red[RED_NG_RESID] = 0.0;
  if (resid) *resid = r;
  if (!isfinite(r)) { *done = 1; atomicOr(errword, ERRBIT_NONFINITE); return; }
  if (eps > 0.0 && r < eps) { *done = 1; return; }
  if (iters) *iters += 1;
}

}  // namespace

void k_prep_coords(const float* Z, const float* X, const float* ell, int M, int Mp, int B, int D,
                   float* Zs, float* Xs, cudaStream_t st, const float* s, double* logs) {
  int Dp = (D + 3) & ~3;
  int tot = (Mp + B) * Dp;
  int grid = (tot + 255) / 256;
  if (grid > 4096) grid = 4096;
  svgp_note_launch();
  pdl_launch(prep_coords_kernel, grid, 256, 0, st, Z, X, ell, M, Mp, B, D, Zs, Xs, s, logs);
}

template <class OutP>
void k_kuu(const float* Zs, int M, int Mp, int D, const float* sf2, float* Kf, OutP Klo, bool has_lo,
           cudaStream_t st) {
  const int nb = Mp / 64;
  dim3 grid(nb * (nb + 1) / 2), blk(32, 8);
  svgp_note_launch();
  SVGP_DP_DISPATCH(D, pdl_launch(kuu_kernel<OutP, DP>, grid, blk, 0, st, Zs, M, Mp, D, sf2, Kf, Klo, has_lo));
}
template void k_kuu<float*>(const float*, int, int, int, const float*, float*, float*, bool, cudaStream_t);
template void k_kuu<bf16*>(const float*, int, int, int, const float*, float*, bf16*, bool, cudaStream_t);
template void k_kuu<SplitPtr>(const float*, int, int, int, const float*, float*, SplitPtr, bool, cudaStream_t);
template void k_kuu<Split3Ptr>(const float*, int, int, int, const float*, float*, Split3Ptr, bool, cudaStream_t);

template <class OutP>
void k_prep_L(const float* Lin, int M, int Mp, float* Lf, OutP Llo, OutP Ltlo, double* logdet, cudaStream_t st) {
  dim3 grid(Mp / 32, Mp / 128), blk(32, 8);
  svgp_note_launch();
  pdl_launch(prep_L_kernel<OutP>, grid, blk, 0, st, Lin, M, Mp, Lf, Llo, Ltlo, logdet);
}
template void k_prep_L<float*>(const float*, int, int, float*, float*, float*, double*, cudaStream_t);
template void k_prep_L<bf16*>(const float*, int, int, float*, bf16*, bf16*, double*, cudaStream_t);
template void k_prep_L<SplitPtr>(const float*, int, int, float*, SplitPtr, SplitPtr, double*, cudaStream_t);

void k_gemv(const float* A, int Mp, int M, const float* x, float alpha, const float* x2, float beta,
            float* y, const float* dotw, double* dot_out, cudaStream_t st) {
  int warps = M, blocks = (warps * 32 + 255) / 256;
  svgp_note_launch();
  pdl_launch(gemv_kernel, blocks, 256, sizeof(float) * Mp, st, A, Mp, M, x, alpha, x2, beta, y, dotw, dot_out);
}

namespace {
struct ZeroList {
  uint32_t* p[ZERO_MAX];
  size_t n[ZERO_MAX];   // 32-bit words
};

__global__ void zero_kernel(ZeroList z) {
  pdl_enter();
  const size_t stride = (size_t)gridDim.x * blockDim.x;
#pragma unroll
  for (int r = 0; r < ZERO_MAX; ++r)
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < z.n[r]; e += stride) z.p[r][e] = 0u;
}

__global__ void kt_f32_kernel(const float* __restrict__ Kuu, const float* __restrict__ s, int M, int Mp,
                              float* __restrict__ Kt) {
  pdl_enter();
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)Mp * Mp) return;
  const int i = (int)(e / Mp), j = (int)(e % Mp);
  Kt[e] = Kuu[e] + ((i == j && i < M) ? s[i] : 0.f);
}

__global__ void gap_check_kernel(const double* __restrict__ red, const float* __restrict__ s, int M,
                                 double sigma2_host, const float* __restrict__ noise, double eps, int* done,
                                 double* gap) {
  pdl_enter();
  __shared__ float mn[32];
  float m = 3.4e38f;
  for (int i = threadIdx.x; i < M; i += blockDim.x) m = fminf(m, s[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) mn[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fminf(m, mn[w]);
  if (done && *done) return;
  const double sig2 = sigma2_host > 0.0 ? sigma2_host : (double)m;
  const double G = red[RED_GAPDOT] / sig2;
  if (gap) *gap = G;
  if (done && eps > 0.0 && G <= 2.0 * (double)*noise * eps) *done = 1;
}

__global__ void axpy_kernel(const float* __restrict__ x, float alpha, const float* __restrict__ x2, float beta,
                            float* __restrict__ y, int n) {
  pdl_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = alpha * (x[i] + beta * x2[i]);
}
}  // namespace

void k_zero_n(cudaStream_t st, const ZeroRange* r, int n) {
  ZeroList z;
  size_t mx = 0;
  for (int k = 0; k < ZERO_MAX; ++k) {
    const bool on = k < n && r[k].p;
    z.p[k] = on ? (uint32_t*)r[k].p : nullptr;
    z.n[k] = on ? r[k].bytes / 4 : 0;
    if (z.n[k] > mx) mx = z.n[k];
  }
  size_t grid = (mx + 255) / 256;
  if (grid < 1) grid = 1;
  if (grid > 1024) grid = 1024;
  svgp_note_launch();
  pdl_launch(zero_kernel, (unsigned)grid, 256, 0, st, z);
}

void k_zero(cudaStream_t st, void* p0, size_t b0, void* p1, size_t b1, void* p2, size_t b2) {
  const ZeroRange r[3] = {{p0, b0}, {p1, b1}, {p2, b2}};
  k_zero_n(st, r, 3);
}

void k_kt_f32(const float* Kuu, const float* s, int M, int Mp, float* Kt, cudaStream_t st) {
  const size_t n = (size_t)Mp * Mp;
  svgp_note_launch();
  pdl_launch(kt_f32_kernel, (unsigned)((n + 255) / 256), 256, 0, st, Kuu, s, M, Mp, Kt);
}

void k_gap_check(const double* red, const float* s, int M, double sigma2_host, const float* noise, double eps,
                 int* done, double* gap, cudaStream_t st) {
  svgp_note_launch();
  pdl_launch(gap_check_kernel, 1, 256, 0, st, red, s, M, sigma2_host, noise, eps, done, gap);
}

void k_axpy(const float* x, float alpha, const float* x2, float beta, float* y, int n, cudaStream_t st) {
  svgp_note_launch();
  pdl_launch(axpy_kernel, (n + 255) / 256, 256, 0, st, x, alpha, x2, beta, y, n);
}

void k_mu(const float* Zs, const float* Xs, int M, int B, int D, const float* sf2, const float* v,
          float* mu, cudaStream_t st) {
  k_zero(st, mu, sizeof(float) * B);
  dim3 grid((B + 511) / 512, (M + 63) / 64);
  svgp_note_launch();
  SVGP_DP_DISPATCH(D, pdl_launch(mu_kernel<DP>, grid, 128, 0, st, Zs, Xs, M, B, D, sf2, v, mu));
}

void k_pointwise_gauss(const float* y, const float* mu, const float* noise, int B, float* g,
                       double* red, cudaStream_t st) {
  int grid = (B + 255) / 256;
  if (grid > 256) grid = 256;
  svgp_note_launch();
  pdl_launch(pointwise_gauss_kernel, grid, 256, 0, st, y, mu, noise, B, g, red);
}

void k_kg(const float* Zs, const float* Xs, int M, int Mp, int B, int D, const float* sf2,
          const float* g, float* Kg, cudaStream_t st) {
  k_zero(st, Kg, sizeof(float) * Mp);
  dim3 grid((M + 511) / 512, (B + 63) / 64);
  svgp_note_launch();
  SVGP_DP_DISPATCH(D, pdl_launch(kg_kernel<DP>, grid, 128, 0, st, Zs, Xs, M, B, D, sf2, g, Kg));
}

template <class OutP>
void k_gp_assemble(const float* Kuu, const float* Psi, const float* Kg, const float* m, const float* w,
                   const float* noise, float c, int M, int Mp, OutP out, cudaStream_t st) {
  dim3 grid((Mp / 4 + 127) / 128, Mp);
  svgp_note_launch();
  pdl_launch(gp_assemble_kernel<OutP>, grid, 128, 0, st, Kuu, Psi, Kg, m, w, noise, c, M, Mp, out);
}
template void k_gp_assemble<float*>(const float*, const float*, const float*, const float*, const float*,
                                    const float*, float, int, int, float*, cudaStream_t);
template void k_gp_assemble<bf16*>(const float*, const float*, const float*, const float*, const float*,
                                   const float*, float, int, int, bf16*, cudaStream_t);
template void k_gp_assemble<SplitPtr>(const float*, const float*, const float*, const float*, const float*,
                                      const float*, float, int, int, SplitPtr, cudaStream_t);

void k_kuu_bwd(const float* GKuu, const float* Kuu, const float* Zs, int M, int Mp, int D,
               float* rowacc_u, double* red, cudaStream_t st) {
  (void)red;
  // One wave: blocks per SM x SMs slots, shared out over the row blocks; JB
  // a multiple of 8, the staged z~ with the static partials within 48 KB.
  SVGP_DP_DISPATCH(D, {
    constexpr int ZW = kuu_zw<DP>();
    const int jbmax = std::min(512, 9216 / ZW);
    static int occ = 0;
    if (!occ) {
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kuu_bwd_kernel<DP>, 256, (size_t)jbmax * ZW * 4);
      if (occ < 1) occ = 1;
    }
    const int gx = (M + 31) / 32;
    const int gy0 = std::max(1, occ * tc_num_sms() / gx);
    int JB = ((M + gy0 - 1) / gy0 + 7) / 8 * 8;
    JB = std::max(8, std::min(JB, jbmax));
    dim3 grid(gx, (M + JB - 1) / JB);
    svgp_note_launch();
    pdl_launch(kuu_bwd_kernel<DP>, grid, 256, (size_t)JB * ZW * 4, st, GKuu, Kuu, Zs, M, Mp, D, rowacc_u, JB);
  });
}

void k_logs(const float* s, int M, double* red, cudaStream_t st) {
  svgp_note_launch();
  pdl_launch(logs_kernel, (M + 255) / 256, 256, 0, st, s, M, red);
}

void k_grad_finalize(const float* rowacc_f, const float* rowacc_u, const float* rowpart, int nparts, int Mp,
                     const float* ell, int M, int D, float* dZ, double* acc_ell, double* red, cudaStream_t st) {
  int grid = (M + 7) / 8;
  svgp_note_launch();
  pdl_launch(grad_finalize_kernel, grid, 256, 0, st, rowacc_f, rowacc_u, rowpart, nparts, Mp, ell, M, D, dZ, acc_ell, red);
}

void k_terms_finalize(const double* red, const double* acc_ell, const float* sf2, const float* noise,
                      const float* ell, int M, int D, int B, double N, bool probit, int hutch_K, double* terms,
                      float* dsf2, float* dnoise, float* dell, int* errword, cudaStream_t st) {
  svgp_note_launch();
  pdl_launch(terms_finalize_kernel, 1, 96, 0, st, red, acc_ell, sf2, noise, ell, M, D, B, N, probit, hutch_K, terms, dsf2, dnoise,
                                          dell, errword);
}

void k_predict_finalize(const float* colsum, const float* sf2, const float* noise, int Ns, int inc,
                        float* var, cudaStream_t st) {
  svgp_note_launch();
  pdl_launch(predict_finalize_kernel, (Ns + 255) / 256, 256, 0, st, colsum, sf2, noise, Ns, inc, var);
}

void k_adam(float* raw, float* cons, const float* grad, float* m1, float* m2, int* step, const float* hyper,
            const float* zbeta1, int M, int D, cudaStream_t st) {
  int n = M * D + D + 2 + 2 * M;
  int grid = (n + 255) / 256;
  if (grid > 1024) grid = 1024;
  svgp_note_launch();
  pdl_launch(adam_kernel, grid, 256, 0, st, raw, cons, grad, m1, m2, step, hyper, zbeta1, M, D);
  svgp_note_launch();
  pdl_launch(step_inc_kernel, 1, 32, 0, st, step);
}

void k_ng_check(double* red, int M, double eps, int* done, int* iters, double* resid, int* errword,
                cudaStream_t st) {
  svgp_note_launch();
  pdl_launch(ng_check_kernel, 1, 32, 0, st, red, M, eps, done, iters, resid, errword);
}
