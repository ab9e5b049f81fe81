// Internal definitions shared by the kernels of the R-SVGP library.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "svgp.h"

#define SVGP_MAXD 32

typedef __nv_bfloat16 bf16;

// Device error word bits (read by svgp_sync_status).
enum { ERRBIT_NONFINITE = 1, ERRBIT_TIMEOUT = 2 };

// Indices of the FP64 reduction slots in the workspace.
enum {
  RED_NG_RESID = 0,   // sum (A - I)^2 of the current NG iterate
  RED_TRA1 = 1,       // tr(A1), A1 = L^T K~ L
  RED_FROA1 = 2,      // ||A1||_F^2
  RED_SPDIAG = 3,     // sum_i s_i P_ii
  RED_PPSI = 4,       // <P, Psi>
  RED_QUAD = 5,       // v^T Kuu v
  RED_LOGDETL = 6,    // sum_i log|L_ii|
  RED_SQERR = 7,      // sum_n (y_n - mu_n)^2
  RED_LOGS = 8,       // sum_i log s_i
  RED_SUMA_F = 9,     // sum (G_Kuf o Kuf)
  RED_SUMA_U = 10,    // sum (G_Kuu o Kuu)
  RED_ELL = 11,       // probit: sum_n E_n
  RED_SUMH = 12,      // probit: sum_n h_n
  RED_SUMVAR = 13,    // probit: sum_n sigma_n^2 (clamped)
  RED_NCLAMP = 14,    // probit: number of clamped sigma_n^2
  RED_GAPDOT = 15,    // <N N^T, Psi> of the Prop. 3 gap
  RED_HKT = 16,       // Hutchinson: sum_k z_k^T L^T K~ L z_k
  RED_HW1 = 17,       // Hutchinson: sum_k z_k^T T Kuu z_k
  RED_HX4 = 18,       // Hutchinson: sum_k z_k^T T K~ T Kuu z_k
  RED_COUNT = 24
};

// One output tile of a GEMM: rows [m0, m0+BM), cols [n0, n0+BN), and the
// K range [k0, k1) that can hold non-zero products (triangular operands).
struct Tile {
  int m0, n0, k0, k1;
};

enum Region { REG_FULL = 0, REG_UPPER = 1, REG_LOWER = 2 };

// Low-precision operand stored as an unevaluated sum hi + lo of two BF16
// matrices (lo = bf16(x - hi)); products use hi*hi + hi*lo + lo*hi.
struct SplitPtr {
  bf16* hi;
  bf16* lo;
};
// three planes, x ~ hi + lo + lo2 (rounding about 2^-26 of |x|)
struct Split3Ptr {
  bf16* hi;
  bf16* lo;
  bf16* lo2;
};

__device__ __forceinline__ void put(float* p, size_t i, float x) { p[i] = x; }
__device__ __forceinline__ void put(bf16* p, size_t i, float x) { p[i] = __float2bfloat16_rn(x); }
__device__ __forceinline__ void put(const SplitPtr& p, size_t i, float x) {
  bf16 h = __float2bfloat16_rn(x);
  p.hi[i] = h;
  p.lo[i] = __float2bfloat16_rn(x - __bfloat162float(h));
}
__device__ __forceinline__ void put(const Split3Ptr& p, size_t i, float x) {
  const bf16 h = __float2bfloat16_rn(x);
  const float r = x - __bfloat162float(h);
  const bf16 l = __float2bfloat16_rn(r);
  p.hi[i] = h;
  p.lo[i] = l;
  p.lo2[i] = __float2bfloat16_rn(r - __bfloat162float(l));
}
// Four consecutive elements from i (a multiple of 4): one vector store per plane.
__device__ __forceinline__ void put4(float* p, size_t i, const float (&x)[4]) {
  *reinterpret_cast<float4*>(p + i) = make_float4(x[0], x[1], x[2], x[3]);
}
__device__ __forceinline__ uint2 bf16x4(float a, float b, float c, float d) {
  __nv_bfloat162 lo = __floats2bfloat162_rn(a, b), hi = __floats2bfloat162_rn(c, d);
  return make_uint2(*reinterpret_cast<uint32_t*>(&lo), *reinterpret_cast<uint32_t*>(&hi));
}
__device__ __forceinline__ void put4(bf16* p, size_t i, const float (&x)[4]) {
  *reinterpret_cast<uint2*>(p + i) = bf16x4(x[0], x[1], x[2], x[3]);
}
__device__ __forceinline__ void put4(const SplitPtr& p, size_t i, const float (&x)[4]) {
  float r[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) r[q] = x[q] - __bfloat162float(__float2bfloat16_rn(x[q]));
  *reinterpret_cast<uint2*>(p.hi + i) = bf16x4(x[0], x[1], x[2], x[3]);
  *reinterpret_cast<uint2*>(p.lo + i) = bf16x4(r[0], r[1], r[2], r[3]);
}

// Reduce a per-thread double over the block and add it to *dst (one atomic
// per block).  Must be called by all threads of the block (any block shape).
// Programmatic dependent launch.  Every kernel of the library starts with
// pdl_enter(): it waits until the kernel launched before it on the stream has
// completed and its memory is visible (a no-op without a programmatic
// dependency), then allows the next kernel to be launched, so that kernel's
// launch and CTA placement overlap this kernel's run.  No kernel touches
// global memory (or allocates TMEM) before the wait.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Packed FP32 pairs (Blackwell f32x2 FMA): two fused multiply-adds per
// instruction, each rounded as fmaf.
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 pack2(float a, float b) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void unpack2(f32x2 v, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ void fma2(f32x2& d, f32x2 a, f32x2 b) {   // d = a * b + d
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(d) : "l"(a), "l"(b));
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}

// Host side: launch `kern` with programmatic stream serialization allowed.
template <typename... KArgs, typename... Args>
inline cudaError_t pdl_launch(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<Args&&>(args)...);
}

__device__ __forceinline__ void block_add_double(double x, double* dst) {
  __shared__ double red_buf[32];
  const unsigned tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const unsigned nthr = blockDim.x * blockDim.y * blockDim.z;
  unsigned lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  __syncthreads();
  if (lane == 0) red_buf[warp] = x;
  __syncthreads();
  if (warp == 0) {
    unsigned nw = (nthr + 31) >> 5;
    double y = lane < nw ? red_buf[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
    if (lane == 0 && y != 0.0) atomicAdd(dst, y);
  }
}

// ---------------------------------------------------------------------------
// GEMM epilogues.  A GEMM mainloop computes acc(i, j) = sum_k A[i,k] B[j,k]
// for its tile and hands it to the epilogue one 32 x 32 block per warp:
//   block(i0, j0, v, vt, lane)   v[q]  = acc(i0 + lane, j0 + q)   (row layout)
//                                vt[r] = acc(i0 + r, j0 + lane)   (column layout)
// Direct writes C[i][j] use the column layout (a warp writes 32 consecutive
// elements of row i0 + r); transposed (mirror) writes C[j][i] use the row
// layout.  Region predicates are applied per element so that every element
// of a symmetric result is produced by exactly one tile.  Every global read
// of an epilogue is issued as a batch of 32 independent loads before any
// store (the compiler cannot reorder loads across stores it cannot prove
// disjoint).  Per-thread partial sums are FP32 (a thread adds at most a few
// hundred terms; FP64 arithmetic is slow on this part) and the block-level
// reduction in reduce() is FP64; every thread of the block calls it.
// ---------------------------------------------------------------------------

// Optional row-layout step of a functor (called before the transpose).
template <class E>
__device__ __forceinline__ auto call_pre(E& e, int i0, int j0, float (&v)[32], int lane, int)
    -> decltype(e.pre(i0, j0, v, lane), void()) {
  e.pre(i0, j0, v, lane);
}
template <class E>
__device__ __forceinline__ void call_pre(E&, int, int, float (&)[32], int, long) {}

// block() with the warp's 32 x 32 shared-memory scratch (row stride lds, odd,
// so row and column accesses are conflict-free) when the functor takes it.
template <class E>
__device__ __forceinline__ auto call_block(E& e, int i0, int j0, const float (&v)[32], const float (&vt)[32], int lane,
                                           float* scr, int lds, int) -> decltype(e.block(i0, j0, v, vt, lane, scr, lds), void()) {
  e.block(i0, j0, v, vt, lane, scr, lds);
}
template <class E>
__device__ __forceinline__ void call_block(E& e, int i0, int j0, const float (&v)[32], const float (&vt)[32], int lane,
                                           float*, int, long) {
  e.block(i0, j0, v, vt, lane);
}

// Vt = L^T K~ = L^T Kuu + L^T diag(s): the diagonal of S~ is added in FP32 so
// that it is not lost when Kuu is rounded (Section 2: S~ lower-bounds the
// eigenvalues of K~).  Lt[i,j] = L[j,i].  s == nullptr: plain L^T S.
template <class OutP>
struct EpiVt {
  OutP out; int ld;
  const float* Lf; const float* s; int M;
  const int* skip_flag;
  __device__ bool skip() const { return skip_flag && *skip_flag; }
  __device__ void begin_tile(int, int) {}
  // Row layout (thread = row i): add Lt[i][j] s[j] = L[j][i] s[j]; the reads
  // L[j0 + q][i0 + lane] are coalesced across the warp.
  __device__ __forceinline__ void pre(int i0, int j0, float (&v)[32], int lane) {
    if (!s) return;
    const int i = i0 + lane;
    float lv[32], sv[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) {
      const int j = j0 + q;
      const bool in = (i < M) && (j < M);
      lv[q] = in ? __ldg(Lf + (size_t)j * ld + i) : 0.f;
      sv[q] = in ? __ldg(s + j) : 0.f;
    }
#pragma unroll
    for (int q = 0; q < 32; ++q) v[q] = fmaf(lv[q], sv[q], v[q]);
  }
  __device__ __forceinline__ void block(int i0, int j0, const float (&)[32], const float (&vt)[32], int lane) {
    const int j = j0 + lane;
#pragma unroll
    for (int r = 0; r < 32; ++r) put(out, (size_t)(i0 + r) * ld + j, vt[r]);
  }
  __device__ void reduce() {}
};

// Symmetric result computed on the upper region (i <= j), mirrored.
//  MODE 0 (NG):  writes Phi^T = triu(A) - 1/2 (I + diag A) (Prop. 1), zero
//                lower part; reduces sum (A - I)^2 (Eq. (8)).
//  MODE 1 (FWD): writes 2I - A1; reduces tr(A1), ||A1||_F^2.
//  MODE 2 (BWD): writes A + I/2 (for T G T + T/2).
template <class OutP, int MODE>
struct EpiSym {
  OutP out; int ld; int M;
  double* red;
  const int* skip_flag;
  float p0, p1;
  __device__ bool skip() const { return skip_flag && *skip_flag; }
  __device__ void begin_tile(int, int) { p0 = 0.f; p1 = 0.f; }
  __device__ __forceinline__ void block(int i0, int j0, const float (&v)[32], const float (&vt)[32], int lane) {
    if (i0 > j0 + 31) return;                    // block entirely below the diagonal
    // direct part (i <= j), column layout: i = i0 + r, j = j0 + lane
    const int j = j0 + lane;
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      const int i = i0 + r;
      if (i > j) continue;
      const float a = vt[r];
      float val;
      if (MODE == 0) val = (i < j) ? a : 0.5f * (a - 1.0f);
      else if (MODE == 1) val = (i == j ? 2.0f : 0.0f) - a;
      else val = a + (i == j ? 0.5f : 0.0f);
      put(out, (size_t)i * ld + j, val);
      if (i < M && j < M) {
        const float w = (i == j) ? 1.f : 2.f;
        if (MODE == 0) { const float e = a - (i == j ? 1.f : 0.f); p0 = fmaf(w * e, e, p0); }
        if (MODE == 1) { if (i == j) p0 += a; p1 = fmaf(w * a, a, p1); }
      }
    }
    // mirror part (j, i) for i < j, row layout: i = i0 + lane, j = j0 + q
    const int i = i0 + lane;
#pragma unroll
    for (int q = 0; q < 32; ++q) {
      const int jj = j0 + q;
      if (i >= jj) continue;
      float val;
      if (MODE == 0) val = 0.0f;
      else if (MODE == 1) val = -v[q];
      else val = v[q];
      put(out, (size_t)jj * ld + i, val);
    }
  }
  __device__ void reduce() {
    if (MODE == 0) block_add_double(p0, red + RED_NG_RESID);
    if (MODE == 1) { block_add_double(p0, red + RED_TRA1); block_add_double(p1, red + RED_FROA1); }
  }
};

// N = I - acc on the valid M x M block, zero in the padding (the matrix
// I - T K~ of the Prop. 3 gap); FP32.
struct EpiIminus {
  float* out; int ld; int M;
  const int* skip_flag;
  __device__ bool skip() const { return skip_flag && *skip_flag; }
  __device__ void begin_tile(int, int) {}
  __device__ __forceinline__ void block(int i0, int j0, const float (&)[32], const float (&vt)[32], int lane) {
    const int j = j0 + lane;
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      const int i = i0 + r;
      out[(size_t)i * ld + j] = (i < M && j < M) ? (i == j ? 1.0f : 0.0f) - vt[r] : 0.0f;
    }
  }
  __device__ void reduce() {}
};

// <acc, Psi> over the valid M x M block, added to *dst (FP64).
struct EpiDotPsi {
  const float* Psi; int ld; int M; double* dst;
  const int* skip_flag;
  float p0;
  __device__ bool skip() const { return skip_flag && *skip_flag; }
  __device__ void begin_tile(int, int) { p0 = 0.f; }
  __device__ __forceinline__ void block(int i0, int j0, const float (&)[32], const float (&vt)[32], int lane) {
    const int j = j0 + lane;
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      const int i = i0 + r;
      if (i < M && j < M) p0 = fmaf(vt[r], __ldg(Psi + (size_t)i * ld + j), p0);
    }
  }
  __device__ void reduce() { block_add_double(p0, dst); }
};

// NG update of L (Prop. 1): acc = (L Phi)_ij on the lower region;
// L_ij <- L_ij - gamma * acc.  The whole launch is skipped when the Frobenius
// stopping rule (Eq. (8), Section 3.3) fired.
struct EpiLupd {
  float* Lf; int ld; float* Lout; int M;
  const float* gamma; const int* done;
  __device__ bool skip() const { return *done != 0; }
  __device__ void begin_tile(int, int) {}
  __device__ __forceinline__ void block(int i0, int j0, const float (&)[32], const float (&vt)[32], int lane) {
    if (j0 > i0 + 31) return;
    const float g = *gamma;
    const int j = j0 + lane;
    float old[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) old[r] = (j <= i0 + r) ? Lf[(size_t)(i0 + r) * ld + j] : 0.f;
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      const int i = i0 + r;
      if (j > i) continue;
      const float Ln = old[r] - g * vt[r];
      Lf[(size_t)i * ld + j] = Ln;
      if (i < M && j < M) Lout[(size_t)i * M + j] = Ln;
    }
  }
  __device__ void reduce() {}
};

// Plain store of a full result.
template <class OutP>
struct EpiStore {
  OutP out; int ld;
  const int* skip_flag;
  __device__ bool skip() const { return skip_flag && *skip_flag; }
  __device__ void begin_tile(int, int) {}
  __device__ __forceinline__ void block(int i0, int j0, const float (&)[32], const float (&vt)[32], int lane) {
#pragma unroll
    for (int r = 0; r < 32; ++r) put(out, (size_t)(i0 + r) * ld + j0 + lane, vt[r]);
  }
  __device__ void reduce() {}
};

// Transposed store of a full result, out[j][i] = acc[i][j] (tensor-core
// path only): the tall-skinny products of the P-free bound keep every M x N
// factor as its transpose, the K-major operand of the next product.
template <class OutP>
struct EpiStoreT {
  OutP out; int ld;
  __device__ bool skip() const { return false; }
  __device__ void begin_tile(int, int) {}
  __device__ void reduce() {}
};

// P = Y L^T = L (2I - A1) L^T on the lower region, mirrored; FP32 and
// low-precision copies; reduces sum_i s_i P_ii and <P, Psi> (Psi may be null).
template <class OutP>
struct EpiP {
  float* Pf; OutP Plo; int ld; int M;
  const float* s; const float* Psi; double* red;
  float p0, p1;
  __device__ bool skip() const { return false; }
  __device__ void begin_tile(int, int) { p0 = 0.f; p1 = 0.f; }
  __device__ __forceinline__ void block(int i0, int j0, const float (&v)[32], const float (&vt)[32], int lane) {
    if (j0 > i0 + 31) return;
    const int j = j0 + lane;
    float ps[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      const int i = i0 + r;
      ps[r] = (Psi && j <= i && i < M && j < M) ? __ldg(Psi + (size_t)i * ld + j) : 0.f;
    }
    const float sj = (j < M) ? __ldg(s + j) : 0.f;
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      const int i = i0 + r;
      if (j > i) continue;
      const float a = vt[r];
      const size_t o = (size_t)i * ld + j;
      Pf[o] = a;
      put(Plo, o, a);
      if (i < M && j < M) {
        if (i == j) p0 = fmaf(sj, a, p0);
        p1 = fmaf((i == j ? 1.f : 2.f) * a, ps[r], p1);
      }
    }
    const int i = i0 + lane;
#pragma unroll
    for (int q = 0; q < 32; ++q) {
      const int jj = j0 + q;
      if (jj >= i) continue;
      const size_t o = (size_t)jj * ld + i;
      Pf[o] = v[q];
      put(Plo, o, v[q]);
    }
  }
  __device__ void reduce() {
    block_add_double(p0, red + RED_SPDIAG);
    if (Psi) block_add_double(p1, red + RED_PPSI);
  }
};

// G_K~ = -L (L^T G_P L + I/2) L^T on the lower region (acc = L S L^T part);
// writes G_Kuu = G_K~ + P/2 - v v^T/2 (symmetric: each value is computed once
// in the column layout, written directly, and written mirrored through the
// warp's shared-memory scratch) and ds_i = G_K~_ii + 1/(2 s_i).
struct EpiGK {
  float* GKuu; int ld; int M;
  const float* Pf; const float* v; const float* s; float* ds;
  __device__ bool skip() const { return false; }
  __device__ void begin_tile(int, int) {}
  __device__ __forceinline__ void block(int i0, int j0, const float (&)[32], const float (&vt)[32], int lane,
                                        float* scr, int lds) {
    if (j0 > i0 + 31) return;
    const int j = j0 + lane;
    const float vj = j < M ? __ldg(v + j) : 0.f;
    const float vrow = (i0 + lane) < M ? __ldg(v + i0 + lane) : 0.f;     // v[i0 + lane], shuffled below
    float pc[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) pc[r] = (j <= i0 + r) ? __ldg(Pf + (size_t)(i0 + r) * ld + j) : 0.f;
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      const int ii = i0 + r;
      const float vi = __shfl_sync(0xffffffffu, vrow, r);
      const float g = -vt[r] + 0.5f * pc[r] - 0.5f * vi * vj;
      scr[r * lds + lane] = g;
      if (j <= ii) GKuu[(size_t)ii * ld + j] = g;
      if (ii == j && ii < M) ds[ii] = -vt[r] + 0.5f / s[ii];
    }
    __syncwarp();
    // mirror: G[j0 + q][i0 + lane] = g(i0 + lane, j0 + q) for j0 + q < i0 + lane
    const int i = i0 + lane;
#pragma unroll
    for (int q = 0; q < 32; ++q) {
      if (j0 + q < i) GKuu[(size_t)(j0 + q) * ld + i] = scr[lane * lds + q];
    }
    __syncwarp();
  }
  __device__ void reduce() {}
};

// Psi = Kuf Kuf^T on the upper region, mirrored (FP32).
struct EpiPsi {
  float* Psi; int ld;
  __device__ bool skip() const { return false; }
  __device__ void begin_tile(int, int) {}
  __device__ __forceinline__ void block(int i0, int j0, const float (&v)[32], const float (&vt)[32], int lane) {
    if (i0 > j0 + 31) return;
    const int j = j0 + lane;
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      const int i = i0 + r;
      if (i <= j) Psi[(size_t)i * ld + j] = vt[r];
    }
    const int i = i0 + lane;
#pragma unroll
    for (int q = 0; q < 32; ++q) {
      const int jj = j0 + q;
      if (i < jj) Psi[(size_t)jj * ld + i] = v[q];
    }
  }
  __device__ void reduce() {}
};

// Parameters of the Kuf generator: scaled coordinates z~ = z / ell (Mp x Dp,
// padded rows and columns zero) and x~ = x / ell (B x Dp), and sf2.  The
// SE-ARD value is sf2 * exp(-1/2 ||z~_i - x~_n||^2).
struct KufGen {
  const float* Zs; const float* Xs; int D; int M; int B; const float* sf2;
};

// Epilogue data for W = P Kuf (the data part of the backward pass): for each
// element A_in = c * Kuf_in * (v_i g_n - 2 h_n W_in) (= G_Kuf o Kuf, with
// g_n = dE_n/dmu_n and h_n = dE_n/dsigma_n^2; hn == null means the Gaussian
// h_n = -1 / (2 noise), so -2 h_n = 1 / noise) accumulates per row i, over
// scaled differences
// e_d = x~_nd - z~_id,
//   rowacc[i][d]     += A_in e_d          (d < D)
//   rowacc[i][D + d] += A_in e_d^2
//   rowacc[i][2D]    += A_in
// and, when colsum != null, colsum[n] += sum_i Kuf_in W_in (for sigma_n^2).
struct WEpi {
  KufGen gen;
  const float* v; const float* g;
  const float* hn;     // per-point h_n (B), or null (Gaussian: from noise)
  const float* noise;
  float c;
  float* rowacc;       // M x (2D+1), may be null
  float* colsum;       // B, may be null
};
