// out[r] += sum_k Kuf(r, k) w_k with the SE-ARD values generated on chip
// (kuf_common.cuh) from the exponent MMA: the predictive mean mu = Kfu v
// (rows = batch points, k = inducing points, Eq. (7) data term) and Kuf g
// (rows = inducing points, k = batch points, the m~ gradient).
//
// Grid: (128-row blocks) x (groups of k-blocks).  Warp roles (320 threads):
// 0 TMA producer (the 128 row-role vectors once, then 64-point k-role tiles
// through a 4-deep ring), 1 TMEM allocator + MMA issuer (exponent MMA
// 128 x 64 x 64 per k-block into one of two TMEM buffers), 2..9 exp2 and the
// weighted row sums (warp w: TMEM lanes 32 (w mod 4) .. +31, one half of the
// 64 columns).  The two halves meet in shared memory; one atomic per row and
// CTA.  All waits are bounded.
#include "common.cuh"
#include "internal.h"
#include "kuf_common.cuh"
#include "tc_common.cuh"

namespace {

using namespace tc;
using namespace kuf;

constexpr int GS = 4;                                     // k-tile ring depth
constexpr int GV_NBAR = 1 + 2 * GS + 4;
constexpr int GV_SMEM = 1024 + GT + GS * CT + 128 * 4 + 8 * GV_NBAR + 64;
constexpr uint32_t GV_TMEM = 128;                         // two 64-column exponent buffers

__global__ void __launch_bounds__(THREADS, 2)
kuf_gemv_kernel(const __grid_constant__ CUtensorMap tmRow, const __grid_constant__ CUtensorMap tmK,
                const float* __restrict__ w, int nk, int nkb, int kb_per_group, float* __restrict__ out, int nrows,
                int* errword) {
  pdl_enter();
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sRow = base;
  unsigned char* ring = base + GT;
  float* comb = reinterpret_cast<float*>(ring + GS * CT);
  uint64_t* bars = reinterpret_cast<uint64_t*>(comb + 128);
  volatile uint32_t* tmem_slot = reinterpret_cast<volatile uint32_t*>(bars + GV_NBAR);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* consumed = abort_flag + 1;
  auto BAR = [&](int idx) { return smem_u32(&bars[idx]); };
  const int B_ROW = 0, B_LD = 1, B_EMPTY = 1 + GS, B_SFULL = 1 + 2 * GS, B_SEMPTY = 3 + 2 * GS;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r0 = blockIdx.x * 128;
  const int kb0 = blockIdx.y * kb_per_group;
  const int kb1 = min(nkb, kb0 + kb_per_group);
  const int nloc = kb1 > kb0 ? kb1 - kb0 : 0;

  if (threadIdx.x == 0) {
    mbar_init(BAR(B_ROW), 1);
    for (int s = 0; s < GS; ++s) {
      mbar_init(BAR(B_LD + s), 1);
      mbar_init(BAR(B_EMPTY + s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(BAR(B_SFULL + b), 1);
      mbar_init(BAR(B_SEMPTY + b), NTW);
    }
    *abort_flag = 0;
    *consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(smem_u32((const void*)tmem_slot), GV_TMEM);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  constexpr uint32_t ID_DIST = idesc_bf16(128, 64);

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    mbar_expect_tx(BAR(B_ROW), GT);
    tma_load_2d(smem_u32(sRow), &tmRow, 0, r0, BAR(B_ROW));
    int issued = 0;
    for (int j = 0; j < nloc; ++j) {
      const int s = j % GS;
      if (!mbar_wait(BAR(B_EMPTY + s), ((j / GS) & 1) ^ 1) || *abort_flag) { *abort_flag = 1; break; }
      mbar_expect_tx(BAR(B_LD + s), CT);
      tma_load_2d(smem_u32(ring + s * CT), &tmK, 0, (kb0 + j) * KB, BAR(B_LD + s));
      issued = j + 1;
    }
    mbar_wait(BAR(B_ROW), 0);
    if (*abort_flag) {
      for (int j = *consumed; j < issued; ++j) mbar_wait(BAR(B_LD + j % GS), (j / GS) & 1);
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    bool ok = mbar_wait(BAR(B_ROW), 0);
    fence_after();
    const uint64_t rd = sw128_desc(smem_u32(sRow));
    for (int j = 0; j < nloc && ok; ++j) {
      const int s = j % GS, b = j & 1;
      if (!mbar_wait(BAR(B_LD + s), (j / GS) & 1)) { ok = false; break; }
      *consumed = j + 1;
      if (!mbar_wait(BAR(B_SEMPTY + b), ((j >> 1) & 1) ^ 1)) { ok = false; break; }
      fence_after();
      const uint64_t kd = sw128_desc(smem_u32(ring + s * CT));
#pragma unroll
      for (int kk = 0; kk < KB / 16; ++kk) {
        const uint64_t o = (uint64_t)(kk * 2);
        mma_bf16(tmem + 64 * b, rd + o, kd + o, ID_DIST, kk != 0);
      }
      mma_commit(BAR(B_SFULL + b));
      mma_commit(BAR(B_EMPTY + s));
    }
    if (!ok) *abort_flag = 1;
  } else if (warp >= 2) {
    // ---------------- exp2 and weighted row sums ----------------
    const int quad = warp & 3, half = (warp - 2) >> 2;
    const int row = quad * 32 + lane, kcol0 = half * 32;
    const uint32_t lane_off = (uint32_t)(quad * 32) << 16;
    float acc = 0.f;
    for (int j = 0; j < nloc; ++j) {
      if (*abort_flag) break;
      const int b = j & 1;
      const int kbase = (kb0 + j) * KB + kcol0;
      float wk[32];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int k = kbase + 4 * q;
        const float4 f = (k + 3 < nk) ? __ldg(reinterpret_cast<const float4*>(w + k)) : make_float4(0.f, 0.f, 0.f, 0.f);
        wk[4 * q] = f.x; wk[4 * q + 1] = f.y; wk[4 * q + 2] = f.z; wk[4 * q + 3] = f.w;
        if (k + 3 >= nk) {
#pragma unroll
          for (int u = 0; u < 4; ++u) wk[4 * q + u] = (k + u < nk) ? __ldg(w + k + u) : 0.f;
        }
      }
      if (!mbar_wait(BAR(B_SFULL + b), (j >> 1) & 1)) { *abort_flag = 1; break; }
      fence_after();
      float t[32];
      tmem_ld32(tmem + lane_off + 64 * b + kcol0, t);
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(BAR(B_SEMPTY + b));
#pragma unroll
      for (int q = 0; q < 32; ++q) acc = fmaf(ex2(t[q]), wk[q], acc);
    }
    if (half == 1) comb[row] = acc;
    asm volatile("bar.sync 1, %0;" ::"n"(32 * NTW) : "memory");
    if (half == 0 && !*abort_flag && r0 + row < nrows && nloc > 0) atomicAdd(out + r0 + row, acc + comb[row]);
  }
  fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) atomicOr(errword, ERRBIT_TIMEOUT);
  if (warp == 1) {
    fence_after();
    tmem_dealloc(tmem, GV_TMEM);
  }
}

}  // namespace

void tc_gemv_init_attributes() {
  cudaFuncSetAttribute(kuf_gemv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, GV_SMEM);
}

bool tc_kuf_gemv(const bf16* Rrole, int nrows, const bf16* Krole, int nk, const float* w, float* out, bool out_zeroed, int* errword,
                 cudaStream_t st) {
  const int rows_p = (nrows + 127) / 128 * 128;
  const int kp = (nk + 63) / 64 * 64;
  CUtensorMap mr, mk;
  if (!tc_make_map(&mr, Rrole, rows_p, 64, 128) || !tc_make_map(&mk, Krole, kp, 64, 64)) return false;
  if (!out_zeroed) k_zero(st, out, sizeof(float) * nrows);
  const int nkb = kp / 64, rb = rows_p / 128;
  // about two CTAs per SM (both resident), at least 4 k-blocks each
  int groups = (2 * tc_num_sms() + rb - 1) / rb;
  if (groups > (nkb + 3) / 4) groups = (nkb + 3) / 4;
  if (groups < 1) groups = 1;
  const int per = (nkb + groups - 1) / groups;
  groups = (nkb + per - 1) / per;
  dim3 grid(rb, groups);
  svgp_note_launch();
  pdl_launch(kuf_gemv_kernel, grid, THREADS, GV_SMEM, st, mr, mk, w, nk, nkb, per, out, nrows, errword);
  return true;
}
