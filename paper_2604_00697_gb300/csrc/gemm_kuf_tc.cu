// tcgen05 contractions whose SE-ARD operand is generated on chip, so Kuf is
// never written to global memory:
//   PSI:  Psi[i, j] = sum_n Kuf[i, n] Kuf[j, n]        (both operands generated)
//   W:    W[i, n]   = sum_k P[i, k] Kuf[k, n]           (P by TMA, Kuf generated)
// with the fused backward / prediction epilogue on W (WEpi).
//
// Generation of a 128 x 64 operand tile G[r, k] = sf2 exp(-1/2 |p_r - q_k|^2)
// (scaled coordinates p, q) per k-block:
//   1. the cross term S = p . q is a small tcgen05 MMA into TMEM, with each
//      coordinate vector split into BF16 hi + lo parts: the row operand holds
//      [hi, hi, lo] and the k operand [hi, lo, hi] along K, so one K <= 64
//      MMA gives hi.hi + hi.lo + lo.hi (about 16 significant bits);
//   2. four transform warps read S from TMEM (one row per thread), form
//      exp2(log2(e) S + c_r + c_k) with the per-point offsets
//      c = -1/2 log2(e) |p|^2 and log2(sf2), and store BF16 (or hi/lo BF16)
//      values into the 128-byte-swizzled operand buffer of the main MMA;
//   3. one thread issues the main tcgen05 MMA on the generated tile(s).
// Warp roles (192 threads): 0 TMA producer, 1 TMEM allocator + MMA issuer,
// 2..5 transform and then epilogue.  All waits are bounded.
#include "common.cuh"
#include "internal.h"
#include "tc_common.cuh"

namespace {

using namespace tc;

constexpr int KB = 64;                        // k-block (one swizzle atom of BF16)
constexpr int GT = 128 * KB * 2;              // 16 KB: 128-row operand tile
constexpr int CT = 64 * KB * 2;               // 8 KB: 64-row coordinate tile
constexpr int EPI_SCR = 4 * 32 * 33 * 4;
constexpr float LOG2E = 1.4426950408889634f;

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
  static constexpr int NBAR = 3 * STAGES + 6;
  static constexpr int SMEM = 1024 + STATIC + STAGES * STAGE + EPI_SCR + 8 * NBAR + 64;
  static constexpr uint32_t TMEM_COLS = KIND == KIND_PSI ? 512 : 256;
  // TMEM columns: accumulator [0,128); S buffers of 64 columns after it
  __host__ __device__ static constexpr uint32_t S_A(int b) { return 128 + 64 * b; }
  __host__ __device__ static constexpr uint32_t S_B(int b) { return KIND == KIND_PSI ? 256 + 64 * b : 128 + 64 * b; }
};

struct KufArgs {
  // per-point constants c = -1/2 log2(e) |p|^2 of the row and k points
  const float* crow_a;   // PSI: z rows (I);  W: unused
  const float* crow_b;   // PSI: z rows (J);  W: x rows (batch)
  const float* ck;       // PSI: x (batch);   W: z (inducing)
  int nrow_a, nrow_b, nk;   // valid counts (rows beyond are zero)
  int nkb;                  // number of k-blocks
  const float* sf2;
  int* errword;
  double* red;              // W: receives sum_n sum_i Kuf_in W_in in RED_KW (may be null)
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

// Transform 64 cross-term values of one row into the generated tile(s).
template <int NSPLIT>
__device__ __forceinline__ void gen_row(const float (&s)[64], float crow, const float* __restrict__ ck, int kbase,
                                        int nk, bool row_ok, unsigned char* hi, unsigned char* lo, int row) {
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    float v[8];
    const float4 c0 = __ldg(reinterpret_cast<const float4*>(ck + kbase + c * 8));
    const float4 c1 = __ldg(reinterpret_cast<const float4*>(ck + kbase + c * 8 + 4));
    const float cc[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int k = kbase + c * 8 + q;
      const float t = fmaf(s[c * 8 + q], LOG2E, crow + cc[q]);
      v[q] = (row_ok && k < nk) ? ex2(t) : 0.f;
    }
    uint4 ph;
    ph.x = pack_bf16(v[0], v[1]);
    ph.y = pack_bf16(v[2], v[3]);
    ph.z = pack_bf16(v[4], v[5]);
    ph.w = pack_bf16(v[6], v[7]);
    const uint32_t off = (uint32_t)(row * 128 + (((c ^ (row & 7)) & 7) << 4));
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
  epi.block(i0, j0, v, vt, lane);
}

// Fused epilogue of W = P Kuf for one accumulator row i over 128 columns n
// (DP: compile-time bound on the padded input dimension).
template <int DP>
__device__ __forceinline__ void w_epilogue(uint32_t tacc, int i, int n0, const WEpi& we, float* colbuf, int lane,
                                           float& kw) {
  const int D = we.gen.D, Dp = (D + 3) & ~3;
  const bool row_ok = i < we.gen.M;
  float z[DP];
#pragma unroll
  for (int d = 0; d < DP; ++d) z[d] = (d < Dp && row_ok) ? we.gen.Zs[(size_t)i * Dp + d] : 0.f;
  float accZ[DP], accL[DP], accS = 0.f;
#pragma unroll
  for (int d = 0; d < DP; ++d) { accZ[d] = 0.f; accL[d] = 0.f; }
  const float lsf2 = log2f(*we.gen.sf2);
  const float inv_noise = we.noise ? 1.0f / *we.noise : 0.f;
  const float vi = (row_ok && we.v) ? we.v[i] : 0.f;
  for (int c = 0; c < 4; ++c) {
    float w[32];
    tmem_ld32(tacc + (uint32_t)(c * 32), w);
#pragma unroll 4
    for (int q = 0; q < 32; ++q) {
      const int n = n0 + c * 32 + q;
      float prod = 0.f;
      if (n < we.gen.B && row_ok) {
        const float* xn = we.gen.Xs + (size_t)n * Dp;
        float e[DP];
        float r2 = 0.f;
#pragma unroll
        for (int d = 0; d < DP; ++d) {
          e[d] = 0.f;
          if (d < Dp) { e[d] = __ldg(xn + d) - z[d]; r2 = fmaf(e[d], e[d], r2); }
        }
        const float kuf = ex2(lsf2 - 0.5f * LOG2E * r2);
        prod = kuf * w[q];
        if (we.rowacc) {
          const float a = we.c * kuf * fmaf(vi, we.g[n], w[q] * inv_noise);
          accS += a;
#pragma unroll
          for (int d = 0; d < DP; ++d) {
            if (d < D) { const float ae = a * e[d]; accZ[d] += ae; accL[d] = fmaf(ae, e[d], accL[d]); }
          }
        }
      }
      kw += prod;
      if (we.colsum) {
        float sv = prod;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sv += __shfl_xor_sync(0xffffffffu, sv, o);
        if (lane == 0) atomicAdd(colbuf + c * 32 + q, sv);
      }
    }
  }
  if (we.rowacc && row_ok) {
    float* ra = we.rowacc + (size_t)i * (2 * D + 1);
#pragma unroll
    for (int d = 0; d < DP; ++d)
      if (d < D) { atomicAdd(ra + d, accZ[d]); atomicAdd(ra + D + d, accL[d]); }
    atomicAdd(ra + 2 * D, accS);
  }
}

template <int KIND, int NSPLIT>
__global__ void __launch_bounds__(192, 1)
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
  uint64_t* bars = reinterpret_cast<uint64_t*>(reinterpret_cast<unsigned char*>(scratch) + EPI_SCR);
  volatile uint32_t* tmem_slot = reinterpret_cast<volatile uint32_t*>(bars + G::NBAR);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* consumed = abort_flag + 1;
  float* colbuf = reinterpret_cast<float*>(scratch);             // W colsum (after the mainloop)
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
      mbar_init(BAR(B_GEN + s), 4);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(BAR(B_SFULL + b), 1);
      mbar_init(BAR(B_SEMPTY + b), 4);
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
    const int quad = warp & 3;
    const int row = quad * 32 + lane;
    const uint32_t lane_off = (uint32_t)(quad * 32) << 16;
    const float lsf2 = log2f(*ka.sf2);
    float crA = 0.f, crB = 0.f;
    bool okA = false, okB = false;
    if (KIND == KIND_PSI) {
      okA = (m0 + row) < ka.nrow_a;
      okB = (n0 + row) < ka.nrow_b;
      crA = lsf2 + (okA ? ka.crow_a[m0 + row] : 0.f);
      crB = lsf2 + (okB ? ka.crow_b[n0 + row] : 0.f);
    } else {
      okB = (n0 + row) < ka.nrow_b;
      crB = lsf2 + (okB ? ka.crow_b[n0 + row] : 0.f);
    }
    for (int kb = 0; kb < nkb; ++kb) {
      if (*abort_flag) break;
      const int s = kb % S, b = kb & 1;
      if (!mbar_wait(BAR(B_SFULL + b), (kb >> 1) & 1)) { *abort_flag = 1; break; }
      fence_after();
      float sa[64], sbv[64];
      {
        float t0[32], t1[32];
        if (KIND == KIND_PSI) {
          tmem_ld32(tmem + lane_off + G::S_A(b), t0);
          tmem_ld32(tmem + lane_off + G::S_A(b) + 32, t1);
#pragma unroll
          for (int q = 0; q < 32; ++q) { sa[q] = t0[q]; sa[32 + q] = t1[q]; }
        }
        if (KIND == KIND_W || !diag) {
          tmem_ld32(tmem + lane_off + G::S_B(b), t0);
          tmem_ld32(tmem + lane_off + G::S_B(b) + 32, t1);
#pragma unroll
          for (int q = 0; q < 32; ++q) { sbv[q] = t0[q]; sbv[32 + q] = t1[q]; }
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(BAR(B_SEMPTY + b));
      // the generated buffers of stage s are free once the main MMA of kb - S finished
      if (!mbar_wait(BAR(B_EMPTY + s), ((kb / S) & 1) ^ 1)) { *abort_flag = 1; break; }
      unsigned char* st = stg + s * G::STAGE;
      const int kbase = kb * KB;
      if (KIND == KIND_PSI) {
        gen_row<NSPLIT>(sa, crA, ka.ck, kbase, ka.nk, okA, st + G::OFF_GA, st + G::OFF_GA + GT, row);
        if (!diag) gen_row<NSPLIT>(sbv, crB, ka.ck, kbase, ka.nk, okB, st + G::OFF_GB, st + G::OFF_GB + GT, row);
      } else {
        gen_row<NSPLIT>(sbv, crB, ka.ck, kbase, ka.nk, okB, st + G::OFF_GB, st + G::OFF_GB + GT, row);
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(BAR(B_GEN + s));
    }
  }
  __syncwarp();

  // ---------------- epilogue (transform warps) ----------------
  float kw = 0.f;
  if (KIND == KIND_W && we.colsum) {
    // colbuf aliases the epilogue scratch: all threads clear it first
    for (int e = threadIdx.x; e < 128; e += blockDim.x) colbuf[e] = 0.f;
  }
  __syncthreads();
  if (warp >= 2) {
    const int quad = warp & 3;
    bool ok = mbar_wait(BAR(B_ACC), 0);
    fence_after();
    if (!ok) *abort_flag = 1;
    if (ok && !*abort_flag) {
      const uint32_t tacc = tmem + ((uint32_t)(quad * 32) << 16);
      if (KIND == KIND_PSI) {
        float* scr = scratch + (warp - 2) * 32 * 33;
        for (int c = 0; c < 4; ++c) {
          float v[32];
          tmem_ld32(tacc + (uint32_t)(c * 32), v);
          epi_block32(epsi, m0 + quad * 32, n0 + c * 32, v, scr, lane);
        }
      } else {
        const int i = m0 + quad * 32 + lane;
        if (we.gen.D <= 4) w_epilogue<4>(tacc, i, n0, we, colbuf, lane, kw);
        else if (we.gen.D <= 8) w_epilogue<8>(tacc, i, n0, we, colbuf, lane, kw);
        else if (we.gen.D <= 16) w_epilogue<16>(tacc, i, n0, we, colbuf, lane, kw);
        else w_epilogue<24>(tacc, i, n0, we, colbuf, lane, kw);
      }
    }
  }
  if (KIND == KIND_W && ka.red) block_add_double(kw, ka.red + RED_KW);
  fence_before();
  __syncthreads();
  if (KIND == KIND_W && we.colsum && threadIdx.x < 128) {
    const int n = n0 + threadIdx.x;
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

// Split coordinates of the Kuf generator: row role [hi, hi, lo], k role
// [hi, lo, hi] (64 BF16 per point, zero padded), and c = -1/2 log2(e) |p|^2.
__global__ void kuf_prep_kernel(const float* __restrict__ P, int n, int npad, int D, bf16* __restrict__ R,
                                bf16* __restrict__ K, float* __restrict__ c) {
  // one row per threadIdx.y (8 rows per block), 64 threads per row
  __shared__ float part_sum[8][2];
  const int Dp = (D + 3) & ~3;
  const int r = blockIdx.x * 8 + threadIdx.y;
  const int d = threadIdx.x;
  const bool live = r < npad;
  const int part = d / D;               // 0, 1, 2 or beyond (padding)
  const bool val = live && r < n && part < 3;
  const float x = val ? P[(size_t)r * Dp + d % D] : 0.f;
  const bf16 hi = __float2bfloat16_rn(x);
  const bf16 lo = __float2bfloat16_rn(x - __bfloat162float(hi));
  const bf16 z = __float2bfloat16_rn(0.f);
  if (live) {
    R[(size_t)r * 64 + d] = val ? (part == 2 ? lo : hi) : z;
    K[(size_t)r * 64 + d] = val ? (part == 1 ? lo : hi) : z;
  }
  float sq = (val && part == 0) ? x * x : 0.f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
  if ((d & 31) == 0) part_sum[threadIdx.y][d >> 5] = sq;
  __syncthreads();
  if (d == 0 && live) c[r] = -0.5f * LOG2E * (part_sum[threadIdx.y][0] + part_sum[threadIdx.y][1]);
}

template <int KIND, int NSPLIT>
void set_kuf_attr() {
  cudaFuncSetAttribute(kuf_tc_kernel<KIND, NSPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       KGeo<KIND, NSPLIT>::SMEM);
}

}  // namespace

void k_kuf_prep(const float* Zs, const float* Xs, int M, int Mp, int B, int Bp, int D, const KufTC& t,
                cudaStream_t st) {
  dim3 blk(64, 8);
  svgp_note_launch();
  kuf_prep_kernel<<<(Mp + 7) / 8, blk, 0, st>>>(Zs, M, Mp, D, t.ZR, t.ZK, t.cz);
  if (Xs && B > 0) {
    svgp_note_launch();
    kuf_prep_kernel<<<(Bp + 7) / 8, blk, 0, st>>>(Xs, B, Bp, D, t.XR, t.XK, t.cx);
  }
}

void tc_kuf_init_attributes() {
  set_kuf_attr<KIND_PSI, 1>();
  set_kuf_attr<KIND_PSI, 3>();
  set_kuf_attr<KIND_W, 1>();
  set_kuf_attr<KIND_W, 3>();
}

bool tc_kuf_supported(int D) { return D >= 1 && 3 * D <= 64 && tc_available(); }

bool tc_psi(const GemmCtx& g, const KufGen& kg, const KufTC& t, int B, EpiPsi e) {
  if (!tc_kuf_supported(kg.D)) return false;
  const int Bp = (B + 127) / 128 * 128;
  CUtensorMap mr, mk;
  if (!tc_make_map(&mr, t.ZR, g.Mp, 64, 128) || !tc_make_map(&mk, t.XK, Bp, 64, 64)) return false;
  KufArgs ka{t.cz, t.cz, t.cx, kg.M, kg.M, B, Bp / KB, kg.sf2, g.err, nullptr};
  WEpi we{};
  svgp_note_launch();
  if (g.split)
    kuf_tc_kernel<KIND_PSI, 3><<<g.nt[TT_PSI], 192, KGeo<KIND_PSI, 3>::SMEM, g.st>>>(mr, mk, mr, mr, g.tt[TT_PSI], ka, e, we);
  else
    kuf_tc_kernel<KIND_PSI, 1><<<g.nt[TT_PSI], 192, KGeo<KIND_PSI, 1>::SMEM, g.st>>>(mr, mk, mr, mr, g.tt[TT_PSI], ka, e, we);
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
  KufArgs ka{t.cz, t.cx, t.cz, we.gen.M, B, we.gen.M, g.Mp / KB, we.gen.sf2, g.err, t.red};
  EpiPsi ep{nullptr, 0};
  dim3 grid(Bp / 128, g.Mp / 128);
  svgp_note_launch();
  if (g.split)
    kuf_tc_kernel<KIND_W, 3><<<grid, 192, KGeo<KIND_W, 3>::SMEM, g.st>>>(mr, mk, mp, mpl, nullptr, ka, ep, we);
  else
    kuf_tc_kernel<KIND_W, 1><<<grid, 192, KGeo<KIND_W, 1>::SMEM, g.st>>>(mr, mk, mp, mpl, nullptr, ka, ep, we);
  return true;
}
