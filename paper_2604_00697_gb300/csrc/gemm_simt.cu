// FP32 SIMT GEMMs ("FP32 plain" form): acc[i,j] = sum_k A[i,k] B[j,k] with both
// operands K-major (row-major with k contiguous), FP32 FMA, no TF32.  Operand
// tiles either come from memory or are generated on the fly from the SE-ARD
// kernel (Kuf never touches global memory).  128x128 output tiles, 16-deep
// k-steps, 256 threads each owning an 8x8 micro-tile.
#include "common.cuh"
#include "internal.h"

namespace {

constexpr int SB = 128;   // tile edge
constexpr int SK = 16;    // k-step
constexpr int SPAD = 4;

// Operand from memory: row-major [rows][ld], k contiguous.
struct MemLoad {
  const float* p; int ld;
  __device__ void init(int) {}
  __device__ __forceinline__ void fetch(int row0, int k0, float (&r)[8]) const {
    int t = threadIdx.x;
    int rr = t >> 2, kk = (t & 3) * 4;
    float4 a = *reinterpret_cast<const float4*>(p + (size_t)(row0 + rr) * ld + k0 + kk);
    float4 b = *reinterpret_cast<const float4*>(p + (size_t)(row0 + rr + 64) * ld + k0 + kk);
    r[0] = a.x; r[1] = a.y; r[2] = a.z; r[3] = a.w;
    r[4] = b.x; r[5] = b.y; r[6] = b.z; r[7] = b.w;
  }
  __device__ __forceinline__ void stash(const float (&r)[8], float (*S)[SB + SPAD]) const {
    int t = threadIdx.x;
    int rr = t >> 2, kk = (t & 3) * 4;
#pragma unroll
    for (int q = 0; q < 4; ++q) { S[kk + q][rr] = r[q]; S[kk + q][rr + 64] = r[4 + q]; }
  }
};

// Operand generated from the SE-ARD kernel: element (row, k) =
// sf2 * exp(-1/2 ||rp_row - kp_k||^2) over scaled coordinates (stride Dp,
// zero padded), zero when row >= nrow or k >= nk; times sqrt|kh_k| when the
// per-k weights kh are given.
struct GenLoad {
  const float* rp; int nrow;   // row points
  const float* kp; int nk;     // k points
  int Dp; const float* sf2;
  const float* kh;             // per-k weights (may be null)
  float c[SVGP_MAXD];
  float lsf2;
  int myrow;
  __device__ void init(int row0) {
    int t = threadIdx.x;
    myrow = row0 + (t & 127);
    lsf2 = logf(*sf2);
#pragma unroll
    for (int d = 0; d < SVGP_MAXD; ++d) c[d] = (d < Dp && myrow < nrow) ? rp[(size_t)myrow * Dp + d] : 0.f;
  }
  __device__ __forceinline__ void fetch(int, int k0, float (&r)[8]) const {
    int t = threadIdx.x;
    int kb = k0 + (t >> 7) * 8;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      int k = kb + q;
      float val = 0.f;
      if (k < nk && myrow < nrow) {
        const float4* x4 = reinterpret_cast<const float4*>(kp + (size_t)k * Dp);
        float r2 = 0.f;
#pragma unroll
        for (int d4 = 0; d4 < SVGP_MAXD / 4; ++d4) {
          if (d4 * 4 < Dp) {
            float4 x = __ldg(x4 + d4);
            float e0 = c[d4 * 4] - x.x, e1 = c[d4 * 4 + 1] - x.y, e2 = c[d4 * 4 + 2] - x.z, e3 = c[d4 * 4 + 3] - x.w;
            r2 = fmaf(e0, e0, r2); r2 = fmaf(e1, e1, r2); r2 = fmaf(e2, e2, r2); r2 = fmaf(e3, e3, r2);
          }
        }
        val = expf(lsf2 - 0.5f * r2);
        if (kh) val *= sqrtf(fabsf(__ldg(kh + k)));
      }
      r[q] = val;
    }
  }
  __device__ __forceinline__ void stash(const float (&r)[8], float (*S)[SB + SPAD]) const {
    int t = threadIdx.x;
    int kb = (t >> 7) * 8, rr = t & 127;
#pragma unroll
    for (int q = 0; q < 8; ++q) S[kb + q][rr] = r[q];
  }
};

struct Smem {
  float A[2][SK][SB + SPAD];
  float B[2][SK][SB + SPAD];
};

template <class LA, class LB>
__device__ __forceinline__ void simt_mainloop(LA& la, LB& lb, int m0, int n0, int kb, int ke,
                                              Smem& sm, float (&acc)[8][8]) {
  int t = threadIdx.x;
  int ty = t >> 4, tx = t & 15;
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[r][c] = 0.f;
  if (kb >= ke) return;
  float ra[8], rb[8];
  la.fetch(m0, kb, ra);
  lb.fetch(n0, kb, rb);
  la.stash(ra, sm.A[0]);
  lb.stash(rb, sm.B[0]);
  __syncthreads();
  int buf = 0;
  for (int k0 = kb; k0 < ke; k0 += SK) {
    bool more = (k0 + SK) < ke;
    if (more) { la.fetch(m0, k0 + SK, ra); lb.fetch(n0, k0 + SK, rb); }
#pragma unroll
    for (int kk = 0; kk < SK; ++kk) {
      float4 a0 = *reinterpret_cast<const float4*>(&sm.A[buf][kk][ty * 4]);
      float4 a1 = *reinterpret_cast<const float4*>(&sm.A[buf][kk][64 + ty * 4]);
      float4 b0 = *reinterpret_cast<const float4*>(&sm.B[buf][kk][tx * 4]);
      float4 b1 = *reinterpret_cast<const float4*>(&sm.B[buf][kk][64 + tx * 4]);
      float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(av[r], bv[c], acc[r][c]);
    }
    if (more) {
      la.stash(ra, sm.A[buf ^ 1]);
      lb.stash(rb, sm.B[buf ^ 1]);
    }
    __syncthreads();
    buf ^= 1;
  }
}


// Stage the 128x128 accumulator tile in shared memory, then hand it to the
// epilogue as 32x32 warp blocks (row and column layouts).
template <class Epi>
__device__ __forceinline__ void simt_epilogue(Epi& epi, int m0, int n0, float (&acc)[8][8], float* T) {
  const int ldT = SB + 1;
  int t = threadIdx.x;
  int ty = t >> 4, tx = t & 15;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    int ii = r < 4 ? ty * 4 + r : 64 + ty * 4 + r - 4;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      int jj = c < 4 ? tx * 4 + c : 64 + tx * 4 + c - 4;
      T[ii * ldT + jj] = acc[r][c];
    }
  }
  __syncthreads();
  epi.begin_tile(m0, n0);
  const int warp = t >> 5, lane = t & 31;
  for (int b = warp; b < 16; b += 8) {
    int bi = b >> 2, bj = b & 3;
    float v[32], vt[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) v[q] = T[(bi * 32 + lane) * ldT + bj * 32 + q];
    call_pre(epi, m0 + bi * 32, n0 + bj * 32, v, lane, 0);
#pragma unroll
    for (int q = 0; q < 32; ++q) T[(bi * 32 + lane) * ldT + bj * 32 + q] = v[q];   // this warp's block only
    __syncwarp();
#pragma unroll
    for (int q = 0; q < 32; ++q) vt[q] = T[(bi * 32 + q) * ldT + bj * 32 + lane];
    call_block(epi, m0 + bi * 32, n0 + bj * 32, v, vt, lane, T + (bi * 32) * ldT + bj * 32, ldT, 0);
  }
  epi.reduce();
}

constexpr size_t SIMT_SMEM = sizeof(float) * SB * (SB + 1) > sizeof(Smem) ? sizeof(float) * SB * (SB + 1) : sizeof(Smem);

template <class Epi, class LA, class LB>
__global__ void __launch_bounds__(256) simt_gemm_tiles(const Tile* __restrict__ tiles, LA la, LB lb,
                                                       Epi epi, int kb_over, int ke_over) {
  pdl_enter();
  if (epi.skip()) return;
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  Smem& sm = *reinterpret_cast<Smem*>(dyn_smem);
  Tile tl = tiles[blockIdx.x];
  int kb = tl.k0, ke = tl.k1;
  if (ke_over > 0) { kb = kb_over; ke = ke_over; }
  la.init(tl.m0);
  lb.init(tl.n0);
  float acc[8][8];
  simt_mainloop(la, lb, tl.m0, tl.n0, kb, ke, sm, acc);
  __syncthreads();
  simt_epilogue(epi, tl.m0, tl.n0, acc, reinterpret_cast<float*>(dyn_smem));
}

// W = P Kuf tile (rows i of P, columns n of the batch) with the fused
// backward/predict epilogue (see WEpi in common.cuh).
__global__ void __launch_bounds__(256) simt_w_kernel(MemLoad la, GenLoad lb, int Mp, WEpi we) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char dyn[];
  Smem& sm = *reinterpret_cast<Smem*>(dyn);
  float* T = reinterpret_cast<float*>(dyn);                  // reused after the mainloop
  const int ldT = SB + 1;
  float* Xs = T + SB * ldT;                                  // staged x~ of the tile columns
  int m0 = blockIdx.y * SB, n0 = blockIdx.x * SB;
  la.init(m0);
  lb.init(n0);
  float acc[8][8];
  simt_mainloop(la, lb, m0, n0, 0, Mp, sm, acc);
  int t = threadIdx.x, ty = t >> 4, tx = t & 15;
  // stage W tile in shared memory (the mainloop ended with __syncthreads)
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    int ii = r < 4 ? ty * 4 + r : 64 + ty * 4 + r - 4;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      int jj = c < 4 ? tx * 4 + c : 64 + tx * 4 + c - 4;
      T[ii * ldT + jj] = acc[r][c];
    }
  }
  const int D = we.gen.D, Dp = (D + 3) & ~3;
  for (int e = t; e < SB * Dp; e += 256) {
    int nn = e / Dp, d = e % Dp;
    int n = n0 + nn;
    Xs[e] = (n < we.gen.B) ? we.gen.Xs[(size_t)n * Dp + d] : 0.f;
  }
  __syncthreads();
  // row pass: thread -> row (t >> 1), half of the columns
  int ii = t >> 1, half = t & 1;
  int i = m0 + ii;
  float z[SVGP_MAXD];
#pragma unroll
  for (int d = 0; d < SVGP_MAXD; ++d) z[d] = (d < Dp && i < we.gen.M) ? we.gen.Zs[(size_t)i * Dp + d] : 0.f;
  float accZ[SVGP_MAXD], accL[SVGP_MAXD], accS = 0.f;
#pragma unroll
  for (int d = 0; d < SVGP_MAXD; ++d) { accZ[d] = 0.f; accL[d] = 0.f; }
  const float lsf2 = logf(*we.gen.sf2);
  const float inv_noise = we.noise ? 1.0f / *we.noise : 0.f;
  const float vi = (i < we.gen.M && we.v) ? we.v[i] : 0.f;
  for (int q = 0; q < 64; ++q) {
    int nn = half * 64 + q;
    int n = n0 + nn;
    float w = T[ii * ldT + nn];
    float prod = 0.f;
    if (n < we.gen.B && i < we.gen.M) {
      float r2 = 0.f;
#pragma unroll
      for (int d = 0; d < SVGP_MAXD; ++d) {
        if (d < Dp) { float e = Xs[nn * Dp + d] - z[d]; r2 = fmaf(e, e, r2); }
      }
      float kuf = expf(lsf2 - 0.5f * r2);
      prod = kuf * w;
      if (we.rowacc) {
        const float hc = we.hn ? -2.0f * we.hn[n] : inv_noise;    // -2 h_n
        float a = we.c * kuf * fmaf(vi, we.g[n], w * hc);
        accS += a;
#pragma unroll
        for (int d = 0; d < SVGP_MAXD; ++d) {
          if (d < D) {
            float e = Xs[nn * Dp + d] - z[d];
            float ae = a * e;
            accZ[d] += ae;
            accL[d] = fmaf(ae, e, accL[d]);
          }
        }
      }
    }
    T[ii * ldT + nn] = prod;
  }
  if (we.rowacc) {
    accS += __shfl_xor_sync(0xffffffffu, accS, 1);
#pragma unroll
    for (int d = 0; d < SVGP_MAXD; ++d) {
      accZ[d] += __shfl_xor_sync(0xffffffffu, accZ[d], 1);
      accL[d] += __shfl_xor_sync(0xffffffffu, accL[d], 1);
    }
    if (half == 0 && i < we.gen.M) {
      float* ra = we.rowacc + (size_t)i * (2 * D + 1);
      for (int d = 0; d < D; ++d) { atomicAdd(ra + d, accZ[d]); atomicAdd(ra + D + d, accL[d]); }
      atomicAdd(ra + 2 * D, accS);
    }
  }
  if (we.colsum) {
    __syncthreads();
    int nn = t & 127, rh = t >> 7;
    float sacc = 0.f;
    for (int r = 0; r < 64; ++r) sacc += T[(rh * 64 + r) * ldT + nn];
    __syncthreads();
    float* tmp = Xs;   // reuse
    if (rh == 1) tmp[nn] = sacc;
    __syncthreads();
    if (rh == 0) {
      int n = n0 + nn;
      if (n < we.gen.B) atomicAdd(we.colsum + n, sacc + tmp[nn]);
    }
  }
}


template <class Epi>
void set_smem_attr() {
  cudaFuncSetAttribute(simt_gemm_tiles<Epi, MemLoad, MemLoad>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)SIMT_SMEM);
}

}  // namespace

// ---------------------------------------------------------------------------
// Host launchers (FP32 path).  All matrices are Mp x Mp with ld = Mp.
// ---------------------------------------------------------------------------
template <class Epi>
void simt_gemm(const GemmCtx& g, int tab, const float* A, const float* B, const Epi& e) {
  MemLoad la{A, g.Mp}, lb{B, g.Mp};
  svgp_note_launch();
  pdl_launch(simt_gemm_tiles<Epi, MemLoad, MemLoad>, g.nt[tab], 256, SIMT_SMEM, g.st, g.tt[tab], la, lb, e, 0, 0);
}

template void simt_gemm<EpiVt<float*>>(const GemmCtx&, int, const float*, const float*, const EpiVt<float*>&);
template void simt_gemm<EpiSym<float*, 0>>(const GemmCtx&, int, const float*, const float*, const EpiSym<float*, 0>&);
template void simt_gemm<EpiSym<float*, 1>>(const GemmCtx&, int, const float*, const float*, const EpiSym<float*, 1>&);
template void simt_gemm<EpiSym<float*, 2>>(const GemmCtx&, int, const float*, const float*, const EpiSym<float*, 2>&);
template void simt_gemm<EpiLupd>(const GemmCtx&, int, const float*, const float*, const EpiLupd&);
template void simt_gemm<EpiStore<float*>>(const GemmCtx&, int, const float*, const float*, const EpiStore<float*>&);
template void simt_gemm<EpiP<float*>>(const GemmCtx&, int, const float*, const float*, const EpiP<float*>&);
template void simt_gemm<EpiGK>(const GemmCtx&, int, const float*, const float*, const EpiGK&);
template void simt_gemm<EpiIminus>(const GemmCtx&, int, const float*, const float*, const EpiIminus&);
template void simt_gemm<EpiDotPsi>(const GemmCtx&, int, const float*, const float*, const EpiDotPsi&);

void simt_psi(const GemmCtx& g, const KufGen& kg, int B, EpiPsi e, const float* hw) {
  int Dp = (kg.D + 3) & ~3;
  GenLoad la{kg.Zs, kg.M, kg.Xs, B, Dp, kg.sf2, hw}, lb{kg.Zs, kg.M, kg.Xs, B, Dp, kg.sf2, hw};
  int Bp = (B + SK - 1) / SK * SK;
  svgp_note_launch();
  pdl_launch(simt_gemm_tiles<EpiPsi, GenLoad, GenLoad>, g.nt[TT_PSI], 256, SIMT_SMEM, g.st, g.tt[TT_PSI], la, lb, e, 0, Bp);
}

void simt_w(const GemmCtx& g, const float* P, const WEpi& we) {
  int Dp = (we.gen.D + 3) & ~3;
  MemLoad la{P, g.Mp};
  GenLoad lb{we.gen.Xs, we.gen.B, we.gen.Zs, we.gen.M, Dp, we.gen.sf2};
  dim3 grid((we.gen.B + SB - 1) / SB, g.Mp / SB);
  size_t smem = sizeof(float) * (SB * (SB + 1) + SB * Dp);
  if (smem < sizeof(Smem)) smem = sizeof(Smem);
  svgp_note_launch();
  pdl_launch(simt_w_kernel, grid, 256, smem, g.st, la, lb, g.Mp, we);
}

void simt_init_attributes() {
  cudaFuncSetAttribute(simt_w_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
  set_smem_attr<EpiVt<float*>>();
  set_smem_attr<EpiSym<float*, 0>>();
  set_smem_attr<EpiSym<float*, 1>>();
  set_smem_attr<EpiSym<float*, 2>>();
  set_smem_attr<EpiLupd>();
  set_smem_attr<EpiStore<float*>>();
  set_smem_attr<EpiP<float*>>();
  set_smem_attr<EpiGK>();
  set_smem_attr<EpiIminus>();
  set_smem_attr<EpiDotPsi>();
  cudaFuncSetAttribute(simt_gemm_tiles<EpiPsi, GenLoad, GenLoad>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)SIMT_SMEM);
}
