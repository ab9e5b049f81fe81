// Shared pieces of the two kernels that generate the SE-ARD cross-covariance
// Kuf on chip (gemm_kuf_tc.cu: Psi = Kuf Kuf^T; gemm_w_tc.cu: W = P Kuf).
//
// Generation of a 128 x 64 operand tile G[r, k] = sf2 exp(-1/2 |p_r - q_k|^2)
// (scaled coordinates p, q) per k-block:
//   1. the whole exponent t = log2(G) is one small tcgen05 MMA into TMEM:
//      with p' = sqrt(log2 e) p and the per-point constants
//      c_r = -1/2 |p'_r|^2 and c_k = -1/2 |q'_k|^2 + log2(sf2),
//        t = p'_r . q'_k + c_r + c_k,
//      where each coordinate vector is split into BF16 hi + lo parts (row
//      operand [hi, hi, lo], k operand [hi, lo, hi], giving hi.hi + hi.lo +
//      lo.hi, about 16 significant bits) and each constant into three BF16
//      parts (24 bits) paired with ones on the other side; padded points carry
//      c = -1e30, so their values come out as exactly 0 (kuf_prep_kernel);
//   2. transform warps read t from TMEM (one row per thread), take exp2 and
//      store BF16 (or hi/lo BF16) values into the 128-byte-swizzled operand
//      buffer of the main MMA (gen32);
//   3. one thread issues the main tcgen05 MMA on the generated tile(s).
#pragma once
#include "common.cuh"
#include "tc_common.cuh"

namespace kuf {

constexpr int KB = 64;                        // k-block (one swizzle atom of BF16)
constexpr int GT = 128 * KB * 2;              // 16 KB: 128-row operand tile
constexpr int CT = 64 * KB * 2;               // 8 KB: 64-row coordinate tile
constexpr int NTW = 8;                        // transform / epilogue warps
constexpr int THREADS = 64 + 32 * NTW;        // + TMA producer warp + MMA warp

__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

// 2^t on the FMA pipe (offloads the MUFU unit): t = j + f with j = rint(t)
// taken by the 1.5 * 2^23 rounding trick and |f| <= 1/2; 2^f from its Taylor
// series sum_k (f ln 2)^k / k! to degree DEG (relative truncation error below
// 3.3e-6 for DEG = 5 and 1.7e-7 for DEG = 6); 2^j enters through the exponent
// field.  t is clamped to >= -125, so underflowing values come out as 2^-125
// instead of 0.
template <int DEG>
__device__ __forceinline__ float ex2_poly(float t) {
  t = fmaxf(t, -125.f);
  const float r = t + 12582912.f;
  const float f = t - (r - 12582912.f);
  float p = DEG >= 6 ? 1.5403530393381606e-4f : 1.3333558146428443e-3f;
  if (DEG >= 6) p = fmaf(p, f, 1.3333558146428443e-3f);
  p = fmaf(p, f, 9.6181291076284772e-3f);
  p = fmaf(p, f, 5.5504108664821580e-2f);
  p = fmaf(p, f, 2.4022650695910071e-1f);
  p = fmaf(p, f, 6.9314718055994531e-1f);
  p = fmaf(p, f, 1.0f);
  const int j = __float_as_int(r) - 0x4B400000;
  return __int_as_float(__float_as_int(p) + (j << 23));
}

// Elements q (of each group of 8 generated values) whose exponential runs on
// the FMA pipe instead of the MUFU unit (a build-time choice; every other
// element, 0x55, measured slower at M = 2048, B = 4096: Psi 0.127 -> 0.145 ms
// in split mode, so the MUFU unit alone takes them by default).
#ifndef SVGP_POLY_MASK
#define SVGP_POLY_MASK 0
#endif
constexpr int POLY_MASK = SVGP_POLY_MASK;

// Transform 32 exponents t[q] (k = kcol0 + q within the k-block) of one row
// into BF16 (hi, and lo = value - hi for NSPLIT = 3) operand values at
// columns kcol0 + q of the 128-byte-swizzled tile(s).
template <int NSPLIT>
__device__ __forceinline__ void gen32(const float (&t)[32], unsigned char* hi, unsigned char* lo, int row, int kcol0) {
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    float v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q)
      v[q] = ((POLY_MASK >> q) & 1) ? ex2_poly<NSPLIT == 3 ? 6 : 5>(t[c * 8 + q]) : ex2(t[c * 8 + q]);
    uint4 ph;
    ph.x = pack_bf16(v[0], v[1]);
    ph.y = pack_bf16(v[2], v[3]);
    ph.z = pack_bf16(v[4], v[5]);
    ph.w = pack_bf16(v[6], v[7]);
    const int chunk = (kcol0 >> 3) + c;
    const uint32_t off = (uint32_t)(row * 128 + (((chunk ^ (row & 7)) & 7) << 4));
    *reinterpret_cast<uint4*>(hi + off) = ph;
    if (NSPLIT == 3) {
      const __nv_bfloat162* hp = reinterpret_cast<const __nv_bfloat162*>(&ph);
      float r[8];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float2 f = __bfloat1622float2(hp[q]);
        r[2 * q] = v[2 * q] - f.x;
        r[2 * q + 1] = v[2 * q + 1] - f.y;
      }
      uint4 pl;
      pl.x = pack_bf16(r[0], r[1]);
      pl.y = pack_bf16(r[2], r[3]);
      pl.z = pack_bf16(r[4], r[5]);
      pl.w = pack_bf16(r[6], r[7]);
      *reinterpret_cast<uint4*>(lo + off) = pl;
    }
  }
}

}  // namespace kuf
