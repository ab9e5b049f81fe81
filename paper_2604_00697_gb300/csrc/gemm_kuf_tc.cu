// tcgen05 contractions whose SE-ARD operand is generated on chip, so Kuf is
// never written to global memory:
//   PSI:  Psi[i, j] = sum_n Kuf[i, n] Kuf[j, n]        (both operands generated)
//   W:    W[i, n]   = sum_k P[i, k] Kuf[k, n]           (P by TMA, Kuf generated)
// with the fused backward / prediction epilogue on W (WEpi).
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
//      c = -1e30, so their values come out as exactly 0;
//   2. the transform warps read t from TMEM (one row per thread), take exp2
//      and store BF16 (or hi/lo BF16) values into the 128-byte-swizzled
//      operand buffer of the main MMA;
//   3. one thread issues the main tcgen05 MMA on the generated tile(s).
// Warp roles (320 threads): 0 TMA producer, 1 TMEM allocator + MMA issuer,
// 2..9 transform and then epilogue (warp w covers TMEM lanes 32 (w mod 4) ..
// +31 and one half of the columns).  All waits are bounded.
#include "common.cuh"
#include "internal.h"
#include "tc_common.cuh"

namespace {

using namespace tc;

constexpr int KB = 64;                        // k-block (one swizzle atom of BF16)
constexpr int GT = 128 * KB * 2;              // 16 KB: 128-row operand tile
constexpr int CT = 64 * KB * 2;               // 8 KB: 64-row coordinate tile
constexpr int NTW = 8;                        // transform / epilogue warps
constexpr int KUF_THREADS = 64 + 32 * NTW;
constexpr int STASH_LD = 129;                 // padded row stride (floats) of the W stash
constexpr int STASH_BYTES = 128 * STASH_LD * 4;
constexpr float SQRT_LOG2E = 1.2011224087864498f;   // sqrt(log2(e))

enum { KIND_PSI = 0, KIND_W = 1 };

template <int KIND, int NSPLIT>
struct KGeo {
  static constexpr int NS = NSPLIT == 3 ? 2 : 1;                         // hi (+lo) planes
  static constexpr int STAGES = NSPLIT == 3 ? 2 : 3;
  // stage: [coord tile CT][P tiles NS*GT (W only)][gen A NS*GT (PSI only)][gen B NS*GT]
  static constexpr int OFF_P = CT;
  static constexpr int OFF_GA = CT + (KIND == KIND_W ? NS * GT : 0);
  static constexpr int OFF_GB = OFF_GA + (KIND == KIND_PSI ? NS * GT : 0);
  static constexpr int STAGE = OFF_GB + NS * GT;
  static constexpr int STATIC = (KIND == KIND_PSI ? 2 : 1) * GT;         // row-coordinate tiles
  // W: FP32 copy of the generated Kuf block whose inducing rows are the output
  // rows (see w_epilogue).  The epilogues stage through the (then idle)
  // pipeline buffers.
  static constexpr int EPI = KIND == KIND_PSI ? 0 : STASH_BYTES;
  static_assert(STAGES * STAGE >= 4 * (256 + 128 * 48) && STAGES * STAGE >= NTW * 32 * 33 * 4, "epilogue staging");
  static constexpr int NBAR = 3 * STAGES + 6;
  static constexpr int SMEM = 1024 + STATIC + STAGES * STAGE + EPI + 8 * NBAR + 64;
  static_assert(SMEM <= 232448, "shared memory budget");
  static constexpr uint32_t TMEM_COLS = KIND == KIND_PSI ? 512 : 256;
  // TMEM columns: accumulator [0,128); S buffers of 64 columns after it
  __host__ __device__ static constexpr uint32_t S_A(int b) { return 128 + 64 * b; }
  __host__ __device__ static constexpr uint32_t S_B(int b) { return KIND == KIND_PSI ? 256 + 64 * b : 128 + 64 * b; }
};

struct KufArgs {
  int nkb;                  // number of k-blocks
  int* errword;
};


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
// the FMA pipe instead of the MUFU unit.
constexpr int POLY_MASK = 0;

// Transform 32 exponents t[q] (k = kcol0 + q within the k-block) of one row
// into BF16 (hi, and lo = value - hi for NSPLIT = 3) operand values at
// columns kcol0 + q of the 128-byte-swizzled tile(s).  When stash != null the
// FP32 values also go to stash[(kcol0 + q) * STASH_LD + row].
template <int NSPLIT>
__device__ __forceinline__ void gen32(const float (&t)[32], unsigned char* hi, unsigned char* lo, int row, int kcol0,
                                      float* stash) {
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    float v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = ((POLY_MASK >> q) & 1) ? ex2_poly<NSPLIT == 3 ? 6 : 5>(t[c * 8 + q]) : ex2(t[c * 8 + q]);
    if (stash) {
#pragma unroll
      for (int q = 0; q < 8; ++q) stash[(kcol0 + c * 8 + q) * STASH_LD + row] = v[q];
    }
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

template <class Epi>
__device__ __forceinline__ void epi_block32(Epi& epi, int i0, int j0, const float (&v)[32], float* scr, int lane) {
  float vt[32];
#pragma unroll
  for (int q = 0; q < 32; ++q) scr[lane * 33 + q] = v[q];
  __syncwarp();
#pragma unroll
  for (int r = 0; r < 32; ++r) vt[r] = scr[r * 33 + lane];
  __syncwarp();
  call_block(epi, i0, j0, v, vt, lane, scr, 33, 0);
}

// Fused epilogue of W = P Kuf for the 128 x 128 output block (rows i = m0 + r,
// columns n = n0 + 0..127), run by the 128 epilogue threads, thread r owning
// accumulator row r.  Kuf_in comes from the FP32 stash the transform filled
// while generating the k-blocks that cover rows [m0, m0 + 128), so nothing is
// recomputed.  Gradient mode (rowacc): with A_in = c Kuf_in (v_i g_n + W_in /
// noise), the sums
//   S0_i = sum_n A_in,  S1_id = sum_n A_in x~_nd,  S2_id = sum_n A_in x~_nd^2
// are accumulated in FP32 from x~ and x~^2 staged in shared memory, and turned
// into the differences form
//   sum_n A_in e_d   = S1 - z~_d S0,
//   sum_n A_in e_d^2 = S2 - 2 z~_d S1 + z~_d^2 S0          (e_d = x~_nd - z~_id)
// before they are added to rowacc.  Variance mode (colsum): colsum[n] +=
// sum_i Kuf_in W_in.  The pipeline stage buffers (free once the accumulator is
// final) hold the staged data.
template <int DP>
__device__ __forceinline__ void w_epilogue(uint32_t tacc, int m0, int n0, int r, int half, const WEpi& we,
                                           const float* __restrict__ stash, float* ebuf, bool ok) {
  constexpr int XW = 2 * DP;
  float* colbuf = ebuf;              // column sums (variance mode)
  float* gq = ebuf + 128;            // g_n
  float* xq = ebuf + 256;            // [128][XW]: x~_n (d < D), then x~_n^2; zero padded
  const int D = we.gen.D, Dp = (D + 3) & ~3, B = we.gen.B;
  const int lane = r & 31, tid = half * 128 + r;
  if (ok) {
    if (we.rowacc) {
      for (int e = tid; e < 128 * DP; e += 32 * NTW) {
        const int n = e / DP, d = e - n * DP;
        const float x = (n0 + n < B && d < D) ? we.gen.Xs[(size_t)(n0 + n) * Dp + d] : 0.f;
        xq[n * XW + d] = x;
        xq[n * XW + DP + d] = x * x;
      }
      if (tid < 128) gq[tid] = (n0 + tid < B) ? we.g[n0 + tid] : 0.f;
    }
    if (tid < 128) colbuf[tid] = 0.f;
  }
  asm volatile("bar.sync 1, %0;" ::"n"(32 * NTW) : "memory");
  if (!ok) return;
  const float* krow = stash + r * STASH_LD;
  if (we.rowacc) {
    const int i = m0 + r;
    const bool row_ok = i < we.gen.M;
    const float inv_noise = 1.0f / *we.noise;
    const float cv = row_ok ? we.c * we.v[i] : 0.f;
    const float cn = we.c * inv_noise;
    float S0 = 0.f, S1[DP], S2[DP];
#pragma unroll
    for (int d = 0; d < DP; ++d) { S1[d] = 0.f; S2[d] = 0.f; }
    for (int ch = 2 * half; ch < 2 * half + 2; ++ch) {
      float w[32];
      tmem_ld32(tacc + (uint32_t)(ch * 32), w);
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const int n = ch * 32 + q;
        const float a = krow[n] * fmaf(cv, gq[n], cn * w[q]);
        S0 += a;
        const float4* xv = reinterpret_cast<const float4*>(xq + n * XW);
#pragma unroll
        for (int d4 = 0; d4 < DP / 4; ++d4) {
          const float4 x = xv[d4], x2 = xv[DP / 4 + d4];
          S1[4 * d4 + 0] = fmaf(a, x.x, S1[4 * d4 + 0]);
          S1[4 * d4 + 1] = fmaf(a, x.y, S1[4 * d4 + 1]);
          S1[4 * d4 + 2] = fmaf(a, x.z, S1[4 * d4 + 2]);
          S1[4 * d4 + 3] = fmaf(a, x.w, S1[4 * d4 + 3]);
          S2[4 * d4 + 0] = fmaf(a, x2.x, S2[4 * d4 + 0]);
          S2[4 * d4 + 1] = fmaf(a, x2.y, S2[4 * d4 + 1]);
          S2[4 * d4 + 2] = fmaf(a, x2.z, S2[4 * d4 + 2]);
          S2[4 * d4 + 3] = fmaf(a, x2.w, S2[4 * d4 + 3]);
        }
      }
    }
    if (row_ok) {
      float* ra = we.rowacc + (size_t)i * (2 * D + 1);
      const float* zi = we.gen.Zs + (size_t)i * Dp;
#pragma unroll
      for (int d = 0; d < DP; ++d) {
        if (d < D) {
          const float z = zi[d];
          atomicAdd(ra + d, fmaf(-z, S0, S1[d]));
          atomicAdd(ra + D + d, fmaf(z, fmaf(z, S0, -2.0f * S1[d]), S2[d]));
        }
      }
      atomicAdd(ra + 2 * D, S0);
    }
  } else if (we.colsum) {
    for (int ch = 2 * half; ch < 2 * half + 2; ++ch) {
      float w[32];
      tmem_ld32(tacc + (uint32_t)(ch * 32), w);
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        float sv = krow[ch * 32 + q] * w[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sv += __shfl_xor_sync(0xffffffffu, sv, o);
        if (lane == 0) atomicAdd(colbuf + ch * 32 + q, sv);
      }
    }
  }
}

template <int KIND, int NSPLIT>
__global__ void __launch_bounds__(KUF_THREADS, 1)
kuf_tc_kernel(const __grid_constant__ CUtensorMap tmRow,     // row-coordinate splits (PSI: z, W: x)
              const __grid_constant__ CUtensorMap tmK,       // k-coordinate splits (PSI: x, W: z)
              const __grid_constant__ CUtensorMap tmP,       // W: P hi
              const __grid_constant__ CUtensorMap tmPl,      // W: P lo
              const Tile* __restrict__ tiles, KufArgs ka, EpiPsi epsi, WEpi we) {
  using G = KGeo<KIND, NSPLIT>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sRowA = base;                                   // PSI: z rows of I;  W: x rows
  unsigned char* sRowB = base + GT;                              // PSI: z rows of J
  unsigned char* stg = base + G::STATIC;
  float* scratch = reinterpret_cast<float*>(stg + G::STAGES * G::STAGE);
  uint64_t* bars = reinterpret_cast<uint64_t*>(reinterpret_cast<unsigned char*>(scratch) + G::EPI);
  volatile uint32_t* tmem_slot = reinterpret_cast<volatile uint32_t*>(bars + G::NBAR);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* consumed = abort_flag + 1;
  float* stash = scratch;                                        // W: Kuf[m0 + r][n0 + n] at r * STASH_LD + n
  constexpr int S = G::STAGES;
  auto BAR = [&](int idx) { return smem_u32(&bars[idx]); };
  const int B_STATIC = 0, B_LD = 1, B_EMPTY = 1 + S, B_GEN = 1 + 2 * S, B_SFULL = 1 + 3 * S, B_SEMPTY = 3 + 3 * S,
            B_ACC = 5 + 3 * S;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int m0, n0;
  if (KIND == KIND_PSI) {
    m0 = tiles[blockIdx.x].m0;
    n0 = tiles[blockIdx.x].n0;
  } else {
    m0 = blockIdx.y * 128;     // rows i of P
    n0 = blockIdx.x * 128;     // batch columns n
  }
  const bool diag = (KIND == KIND_PSI) && (m0 == n0);
  const int nkb = ka.nkb;

  if (threadIdx.x == 0) {
    mbar_init(BAR(B_STATIC), 1);
    for (int s = 0; s < S; ++s) {
      mbar_init(BAR(B_LD + s), 1);
      mbar_init(BAR(B_EMPTY + s), 1);
      mbar_init(BAR(B_GEN + s), NTW);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(BAR(B_SFULL + b), 1);
      mbar_init(BAR(B_SEMPTY + b), NTW);
    }
    mbar_init(BAR(B_ACC), 1);
    *abort_flag = 0;
    *consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(smem_u32((const void*)tmem_slot), G::TMEM_COLS);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  constexpr uint32_t ID_MAIN = idesc_bf16(128, 128);
  constexpr uint32_t ID_DIST = idesc_bf16(128, 64);

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    const uint32_t sb = BAR(B_STATIC);
    if (KIND == KIND_PSI) {
      mbar_expect_tx(sb, diag ? GT : 2 * GT);
      tma_load_2d(smem_u32(sRowA), &tmRow, 0, m0, sb);
      if (!diag) tma_load_2d(smem_u32(sRowB), &tmRow, 0, n0, sb);
    } else {
      mbar_expect_tx(sb, GT);
      tma_load_2d(smem_u32(sRowA), &tmRow, 0, n0, sb);
    }
    int issued = 0;
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % S;
      const uint32_t ph = (kb / S) & 1;
      if (!mbar_wait(BAR(B_EMPTY + s), ph ^ 1)) { *abort_flag = 1; break; }
      if (*abort_flag) break;
      unsigned char* st = stg + s * G::STAGE;
      const uint32_t fb = BAR(B_LD + s);
      mbar_expect_tx(fb, CT + (KIND == KIND_W ? G::NS * GT : 0));
      tma_load_2d(smem_u32(st), &tmK, 0, kb * KB, fb);
      if (KIND == KIND_W) {
        tma_load_2d(smem_u32(st + G::OFF_P), &tmP, kb * KB, m0, fb);
        if (NSPLIT == 3) tma_load_2d(smem_u32(st + G::OFF_P + GT), &tmPl, kb * KB, m0, fb);
      }
      issued = kb + 1;
    }
    mbar_wait(sb, 0);
    if (*abort_flag) {
      for (int kb = *consumed; kb < issued; ++kb) mbar_wait(BAR(B_LD + kb % S), (kb / S) & 1);
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    bool ok = mbar_wait(BAR(B_STATIC), 0);
    auto main_mma = [&](int j) -> bool {
      const int s = j % S;
      if (!mbar_wait(BAR(B_GEN + s), (j / S) & 1)) return false;
      fence_after();
      unsigned char* st = stg + s * G::STAGE;
      uint64_t ad, adl, bd, bdl;
      if (KIND == KIND_PSI) {
        ad = sw128_desc(smem_u32(st + G::OFF_GA));
        adl = sw128_desc(smem_u32(st + G::OFF_GA + GT));
        bd = diag ? ad : sw128_desc(smem_u32(st + G::OFF_GB));
        bdl = diag ? adl : sw128_desc(smem_u32(st + G::OFF_GB + GT));
      } else {
        ad = sw128_desc(smem_u32(st + G::OFF_P));
        adl = sw128_desc(smem_u32(st + G::OFF_P + GT));
        bd = sw128_desc(smem_u32(st + G::OFF_GB));
        bdl = sw128_desc(smem_u32(st + G::OFF_GB + GT));
      }
#pragma unroll
      for (int kk = 0; kk < KB / 16; ++kk) {
        const uint64_t o = (uint64_t)(kk * 2);
        mma_bf16(tmem, ad + o, bd + o, ID_MAIN, (j | kk) != 0);
        if (NSPLIT == 3) {
          mma_bf16(tmem, ad + o, bdl + o, ID_MAIN, 1);
          mma_bf16(tmem, adl + o, bd + o, ID_MAIN, 1);
        }
      }
      mma_commit(BAR(B_EMPTY + s));
      return true;
    };
    int done_main = 0;
    for (int kb = 0; kb < nkb && ok; ++kb) {
      const int s = kb % S, b = kb & 1;
      if (!mbar_wait(BAR(B_LD + s), (kb / S) & 1)) { ok = false; break; }
      *consumed = kb + 1;
      if (!mbar_wait(BAR(B_SEMPTY + b), ((kb >> 1) & 1) ^ 1)) { ok = false; break; }
      fence_after();
      unsigned char* st = stg + s * G::STAGE;
      const uint64_t kd = sw128_desc(smem_u32(st));
      const uint64_t ra = sw128_desc(smem_u32(sRowA));
      const uint64_t rb = sw128_desc(smem_u32(sRowB));
#pragma unroll
      for (int kk = 0; kk < KB / 16; ++kk) {
        const uint64_t o = (uint64_t)(kk * 2);
        if (KIND == KIND_PSI) {
          mma_bf16(tmem + G::S_A(b), ra + o, kd + o, ID_DIST, kk != 0);
          if (!diag) mma_bf16(tmem + G::S_B(b), rb + o, kd + o, ID_DIST, kk != 0);
        } else {
          mma_bf16(tmem + G::S_B(b), ra + o, kd + o, ID_DIST, kk != 0);
        }
      }
      mma_commit(BAR(B_SFULL + b));
      if (kb >= 1) {
        if (!main_mma(kb - 1)) { ok = false; break; }
        done_main = kb;
      }
    }
    if (ok && nkb > 0) ok = main_mma(nkb - 1);
    (void)done_main;
    if (!ok) *abort_flag = 1;
    mma_commit(BAR(B_ACC));
  } else if (warp >= 2) {
    // ---------------- transform ----------------
    // warp (quad, half): TMEM lanes / tile rows quad*32 .. +31, k columns half*32 .. +31
    const int quad = warp & 3, half = (warp - 2) >> 2;
    const int row = quad * 32 + lane, kcol0 = half * 32;
    const uint32_t lane_off = (uint32_t)(quad * 32) << 16;
    for (int kb = 0; kb < nkb; ++kb) {
      if (*abort_flag) break;
      const int s = kb % S, b = kb & 1;
      if (!mbar_wait(BAR(B_SFULL + b), (kb >> 1) & 1)) { *abort_flag = 1; break; }
      fence_after();
      float sa[32], sbv[32];
      if (KIND == KIND_PSI) tmem_ld32(tmem + lane_off + G::S_A(b) + kcol0, sa);
      if (KIND == KIND_W || !diag) tmem_ld32(tmem + lane_off + G::S_B(b) + kcol0, sbv);
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(BAR(B_SEMPTY + b));
      // the generated buffers of stage s are free once the main MMA of kb - S finished
      if (!mbar_wait(BAR(B_EMPTY + s), ((kb / S) & 1) ^ 1)) { *abort_flag = 1; break; }
      unsigned char* st = stg + s * G::STAGE;
      if (KIND == KIND_PSI) {
        gen32<NSPLIT>(sa, st + G::OFF_GA, st + G::OFF_GA + GT, row, kcol0, nullptr);
        if (!diag) gen32<NSPLIT>(sbv, st + G::OFF_GB, st + G::OFF_GB + GT, row, kcol0, nullptr);
      } else {
        // the k-blocks covering the output rows [m0, m0 + 128) also fill the stash
        const int kb0 = kb * KB;
        float* sh = (kb0 >= m0 && kb0 < m0 + 128) ? stash + (size_t)(kb0 - m0) * STASH_LD : nullptr;
        gen32<NSPLIT>(sbv, st + G::OFF_GB, st + G::OFF_GB + GT, row, kcol0, sh);
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(BAR(B_GEN + s));
    }
  }
  __syncwarp();

  // ---------------- epilogue (transform warps) ----------------
  if (warp >= 2) {
    const int quad = warp & 3;
    bool ok = mbar_wait(BAR(B_ACC), 0);
    fence_after();
    if (!ok) *abort_flag = 1;
    ok = ok && !*abort_flag;
    const uint32_t tacc = tmem + ((uint32_t)(quad * 32) << 16);
    const int half = (warp - 2) >> 2;
    if (KIND == KIND_PSI) {
      if (ok) {
        float* scr = reinterpret_cast<float*>(stg) + (warp - 2) * 32 * 33;
        for (int c = 2 * half; c < 2 * half + 2; ++c) {
          float v[32];
          tmem_ld32(tacc + (uint32_t)(c * 32), v);
          epi_block32(epsi, m0 + quad * 32, n0 + c * 32, v, scr, lane);
        }
      }
    } else {
      const int r = quad * 32 + lane;
      float* ebuf = reinterpret_cast<float*>(stg);
      if (we.gen.D <= 4) w_epilogue<4>(tacc, m0, n0, r, half, we, stash, ebuf, ok);
      else if (we.gen.D <= 8) w_epilogue<8>(tacc, m0, n0, r, half, we, stash, ebuf, ok);
      else if (we.gen.D <= 16) w_epilogue<16>(tacc, m0, n0, r, half, we, stash, ebuf, ok);
      else w_epilogue<24>(tacc, m0, n0, r, half, we, stash, ebuf, ok);
    }
  }
  fence_before();
  __syncthreads();
  if (KIND == KIND_W && we.colsum && threadIdx.x < 128 && !*abort_flag) {
    const int n = n0 + threadIdx.x;
    const float* colbuf = reinterpret_cast<const float*>(stg);
    if (n < we.gen.B) atomicAdd(we.colsum + n, colbuf[threadIdx.x]);
  }
  if (threadIdx.x == 0 && *abort_flag) atomicOr(ka.errword, ERRBIT_TIMEOUT);
  if (warp == 1) {
    fence_after();
    tmem_dealloc(tmem, G::TMEM_COLS);
  }
}

}  // namespace

namespace {

// Operand vectors of the exponent MMA (64 BF16 per point, zero padded) for
// points p (scaled coordinates, n valid rows of npad):
//   row role R = [p'hi (D), p'hi (D), p'lo (D), c_hi, c_mid, c_lo, 1, 1, 1]
//   k role   K = [p'hi (D), p'lo (D), p'hi (D), 1, 1, 1, c'_hi, c'_mid, c'_lo]
// with p' = sqrt(log2 e) p, c = -1/2 |p'|^2 and c' = c + log2(sf2); padded
// rows get c = c' = -1e30.  R_a . K_b = t(a, b) = log2 of the SE-ARD value.
__global__ void kuf_prep_kernel(const float* __restrict__ P, int n, int npad, int D, const float* __restrict__ sf2,
                                bf16* __restrict__ R, bf16* __restrict__ K) {
  // one row per threadIdx.y (8 rows per block), 64 threads per row
  __shared__ float part_sum[8][2];
  const int Dp = (D + 3) & ~3;
  const int r = blockIdx.x * 8 + threadIdx.y;
  const int d = threadIdx.x;
  const bool live = r < npad, valid = r < n;
  const int part = d / D;               // 0, 1, 2: coordinate slots; then constants
  const float x = (valid && part < 3) ? SQRT_LOG2E * P[(size_t)r * Dp + d % D] : 0.f;
  const bf16 hi = __float2bfloat16_rn(x);
  const bf16 lo = __float2bfloat16_rn(x - __bfloat162float(hi));
  float sq = (part == 0) ? x * x : 0.f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
  if ((d & 31) == 0) part_sum[threadIdx.y][d >> 5] = sq;
  __syncthreads();
  if (!live) return;
  const float c_row = valid ? -0.5f * (part_sum[threadIdx.y][0] + part_sum[threadIdx.y][1]) : -1e30f;
  const float c_k = valid ? c_row + log2f(*sf2) : -1e30f;
  // three-way BF16 split of a constant: component q of (hi, mid, lo)
  auto split3 = [](float c, int q) {
    const float h = __bfloat162float(__float2bfloat16_rn(c));
    const float m = __bfloat162float(__float2bfloat16_rn(c - h));
    return q == 0 ? h : (q == 1 ? m : c - h - m);
  };
  const bf16 one = __float2bfloat16_rn(1.f), z = __float2bfloat16_rn(0.f);
  bf16 rv = z, kv = z;
  if (part < 3) {
    rv = part == 2 ? lo : hi;
    kv = part == 1 ? lo : hi;
  } else if (d < 3 * D + 3) {
    rv = __float2bfloat16_rn(split3(c_row, d - 3 * D));
    kv = one;
  } else if (d < 3 * D + 6) {
    rv = one;
    kv = __float2bfloat16_rn(split3(c_k, d - 3 * D - 3));
  }
  R[(size_t)r * 64 + d] = rv;
  K[(size_t)r * 64 + d] = kv;
}

template <int KIND, int NSPLIT>
void set_kuf_attr() {
  cudaFuncSetAttribute(kuf_tc_kernel<KIND, NSPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       KGeo<KIND, NSPLIT>::SMEM);
}

}  // namespace

void k_kuf_prep(const float* Zs, const float* Xs, int M, int Mp, int B, int Bp, int D, const float* sf2,
                const KufTC& t, cudaStream_t st) {
  dim3 blk(64, 8);
  svgp_note_launch();
  kuf_prep_kernel<<<(Mp + 7) / 8, blk, 0, st>>>(Zs, M, Mp, D, sf2, t.ZR, t.ZK);
  if (Xs && B > 0) {
    svgp_note_launch();
    kuf_prep_kernel<<<(Bp + 7) / 8, blk, 0, st>>>(Xs, B, Bp, D, sf2, t.XR, t.XK);
  }
}

void tc_kuf_init_attributes() {
  set_kuf_attr<KIND_PSI, 1>();
  set_kuf_attr<KIND_PSI, 3>();
  set_kuf_attr<KIND_W, 1>();
  set_kuf_attr<KIND_W, 3>();
}

bool tc_kuf_supported(int D) { return D >= 1 && 3 * D + 6 <= 64 && tc_available(); }

bool tc_psi(const GemmCtx& g, const KufGen& kg, const KufTC& t, int B, EpiPsi e) {
  if (!tc_kuf_supported(kg.D)) return false;
  const int Bp = (B + 127) / 128 * 128;
  CUtensorMap mr, mk;
  if (!tc_make_map(&mr, t.ZR, g.Mp, 64, 128) || !tc_make_map(&mk, t.XK, Bp, 64, 64)) return false;
  KufArgs ka{Bp / KB, g.err};
  WEpi we{};
  svgp_note_launch();
  if (g.split)
    kuf_tc_kernel<KIND_PSI, 3><<<g.nt[TT_PSI], KUF_THREADS, KGeo<KIND_PSI, 3>::SMEM, g.st>>>(mr, mk, mr, mr, g.tt[TT_PSI], ka, e, we);
  else
    kuf_tc_kernel<KIND_PSI, 1><<<g.nt[TT_PSI], KUF_THREADS, KGeo<KIND_PSI, 1>::SMEM, g.st>>>(mr, mk, mr, mr, g.tt[TT_PSI], ka, e, we);
  return true;
}

bool tc_w(const GemmCtx& g, const bf16* P, const KufTC& t, const WEpi& we) {
  if (!tc_kuf_supported(we.gen.D)) return false;
  const int B = we.gen.B;
  const int Bp = (B + 127) / 128 * 128;
  CUtensorMap mr, mk, mp, mpl;
  if (!tc_make_map(&mr, t.XR, Bp, 64, 128) || !tc_make_map(&mk, t.ZK, g.Mp, 64, 64) ||
      !tc_make_map(&mp, P, g.Mp, g.Mp, 128))
    return false;
  if (g.split) {
    if (!tc_make_map(&mpl, P + (size_t)g.Mp * g.Mp, g.Mp, g.Mp, 128)) return false;
  } else {
    mpl = mp;
  }
  KufArgs ka{g.Mp / KB, g.err};
  EpiPsi ep{nullptr, 0};
  dim3 grid(Bp / 128, g.Mp / 128);
  svgp_note_launch();
  if (g.split)
    kuf_tc_kernel<KIND_W, 3><<<grid, KUF_THREADS, KGeo<KIND_W, 3>::SMEM, g.st>>>(mr, mk, mp, mpl, nullptr, ka, ep, we);
  else
    kuf_tc_kernel<KIND_W, 1><<<grid, KUF_THREADS, KGeo<KIND_W, 1>::SMEM, g.st>>>(mr, mk, mp, mpl, nullptr, ka, ep, we);
  return true;
}
