// W = P Kuf with the SE-ARD operand generated on chip (kuf_common.cuh) and a
// fused epilogue, for the data part of the backward pass (Section 3.1) and
// for the predictive variance:
//   gradient mode (rowpart != null): with A_in = c Kuf_in (v_i g_n - 2 h_n
//     W_in) (= G_Kuf o Kuf; h_n = -1/(2 noise) for the Gaussian likelihood,
//     per point for probit), per row i the sums
//       S0 = sum_n A_in,  S1_d = sum_n A_in x~_nd,  S2_d = sum_n A_in x~_nd^2
//     (FP32 in registers; each x~ row staged in shared memory serves a group
//     of four lanes, which exchange their rows' A values by shuffles and
//     split the dimensions among them), reported in the
//     difference form  sum_n A_in e_d = S1_d - z~_id S0  and
//     sum_n A_in e_d^2 = S2_d - 2 z~_id S1_d + z~_id^2 S0  (e_d = x~_nd - z~_id);
//   variance mode (colsum != null): colsum[n] += sum_i Kuf_in W_in.
//
// Grid: (groups of n-blocks) x (row blocks of NI x 128 rows i of P).  A CTA
// keeps its rows i and walks the n-blocks nb = blockIdx.x, blockIdx.x +
// gridDim.x, ..., carrying the row sums in registers; at the end it writes one
// partial row set rowpart[blockIdx.x][k][i] (no atomics; the gradient
// finalize adds the gridDim.x partials).  Per n-block:
//   * mainloop over the inducing k-blocks: exponent MMA for the 128 x 64 block
//     Kuf^T[n, k], exp2 into the swizzled B operand, main MMAs
//     W[i, n] += P[i, k] Kuf[k, n] for each of the NI 128-row blocks: with
//     NI = 2 (BF16 operands) one generated tile feeds two accumulators, which
//     halves the exps per output;
//   * one more exponent MMA per row block, T[i, n] = log2 Kuf_in for the
//     epilogue (z rows of the block against the n-block), so Kuf_in is
//     recomputed exactly as the generator computes it.  Its operands (z rows
//     in row role, x of the n-block in k role) are copied, once the n-block's
//     main MMAs are done, into the generated ring, which is idle then; the
//     shared memory they would hold through the mainloop goes to the TMA
//     ring instead.
// Warp roles (320 threads): 0 TMA producer, 1 TMEM allocator + MMA issuer,
// 2..9 transform and then epilogue (warp w covers TMEM lanes 32 (w mod 4) ..
// +31 and one half of the columns).  All waits are bounded; once a wait has
// timed out the warps skip their work but still pass every named barrier.
#include "common.cuh"
#include "internal.h"
#include "kuf_common.cuh"
#include "tc_common.cuh"

namespace {

using namespace tc;
using namespace kuf;

constexpr int DPMAX = 24;                      // padded-dimension bound of the staged x~ rows

template <int NSPLIT, int NI>
struct WGeo {
  static_assert(NI == 1 || (NI == 2 && NSPLIT == 1), "two row blocks only with BF16 operands");
  static constexpr int NS = NSPLIT == 3 ? 2 : 1;                         // hi (+lo) planes
  // Two rings.  TMA ring, ST stages of [z k-role coordinate tile CT][P tiles
  // NI*NS*GT]: a stage is refilled once the main MMA of its k-block is done,
  // so the copies run ST - 1 k-blocks ahead.  Generated ring, SG stages of
  // Kuf^T tiles NS*GT written by the transform warps (the transform of k-block
  // g + 1 overlaps the main MMA of k-block g).  Cycle stamps of the version
  // with two TMA stages (split operands, M = 2048, B = 4096): one main MMA per
  // 1630 cycles against 768 of MMA work, paced by the copies (a copy waited
  // for the main MMA two k-blocks back, then 1400 cycles to the exponent
  // MMA); one generated stage with three TMA stages measured slower.
  static constexpr int ST = NSPLIT == 3 ? 3 : (NI == 2 ? 3 : 4);
  static constexpr int SG = (NSPLIT == 1 && NI == 2) ? 3 : 2;
  static constexpr int OFF_P = CT;
  static constexpr int TSTAGE = CT + NI * NS * GT;
  static constexpr int GSTAGE = NS * GT;
  // static tile: x rows of the n-block in row role (generator); the epilogue
  // exponent's operands -- z rows of the row blocks in row role, then x of the
  // n-block in k role -- take the start of the generated ring after the
  // mainloop
  static constexpr int OFF_XR = 0, STATIC = GT;
  static_assert(SG * NS * GT >= (NI + 1) * GT, "epilogue exponent operands fit the generated ring");
  // epilogue floats: colbuf[128], gq[128], xq[128][XW <= DPMAX]; from the
  // start, the final combination of the two column halves (128 x (2 DP + 1))
  static constexpr int EPI_FLOATS = 128 * (2 * DPMAX + 1);
  static_assert(EPI_FLOATS >= 256 + 128 * DPMAX, "x~ staging");
  static constexpr int NBAR = 2 * ST + 2 * SG + 9;
  static constexpr int SMEM = 1024 + STATIC + ST * TSTAGE + SG * GSTAGE + 4 * EPI_FLOATS + 8 * NBAR + 64;
  static_assert(SMEM <= 232448, "shared memory budget");
  static constexpr uint32_t TMEM_COLS = 512;
  // TMEM columns: W accumulators [0, 128 NI), generator exponents 2 x 64 after
  // them, epilogue exponents T of row block 0 in [384, 512) and of row block 1
  // in the generator buffers (free once the mainloop of the n-block is done)
  __host__ __device__ static constexpr uint32_t ACC(int ib) { return 128 * ib; }
  __host__ __device__ static constexpr uint32_t SB(int b) { return 128 * NI + 64 * b; }
  __host__ __device__ static constexpr uint32_t T(int ib) { return ib == 0 ? 384 : 128 * NI; }
};

struct WArgs {
  int nkb;          // inducing k-blocks (Mp / 64)
  int nblk;         // n-blocks (Bp / 128)
  int Mp;
  int* errword;
  float* rowpart;   // gradient mode: [gridDim.x][2D + 1][Mp]
};

template <int NSPLIT, int DP, int NI>
__global__ void __launch_bounds__(THREADS, 1)
w_tc_kernel(const __grid_constant__ CUtensorMap tmZR, const __grid_constant__ CUtensorMap tmZK,
            const __grid_constant__ CUtensorMap tmXR, const __grid_constant__ CUtensorMap tmXK,
            const __grid_constant__ CUtensorMap tmP, const __grid_constant__ CUtensorMap tmPl, WArgs wa, WEpi we) {
  pdl_enter();
  using G = WGeo<NSPLIT, NI>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sXR = base + G::OFF_XR;
  unsigned char* stgT = base + G::STATIC;                         // TMA ring
  unsigned char* stgG = stgT + G::ST * G::TSTAGE;                 // generated ring
  float* ebuf = reinterpret_cast<float*>(stgG + G::SG * G::GSTAGE);
  uint64_t* bars = reinterpret_cast<uint64_t*>(ebuf + G::EPI_FLOATS);
  volatile uint32_t* tmem_slot = reinterpret_cast<volatile uint32_t*>(bars + G::NBAR);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* consumed = abort_flag + 1;
  constexpr int ST = G::ST, SG = G::SG;
  auto BAR = [&](int idx) { return smem_u32(&bars[idx]); };
  // LD / TEMPTY: TMA stage landed / free; GEN / GEMPTY: generated stage written / free;
  // MDONE: the n-block's main MMAs completed; ZX: the epilogue exponent's operands landed
  const int B_ZX = 0, B_TILE = 1, B_LD = 2, B_TEMPTY = 2 + ST, B_GEN = 2 + 2 * ST, B_GEMPTY = 2 + 2 * ST + SG,
            B_SFULL = 2 + 2 * ST + 2 * SG, B_SEMPTY = B_SFULL + 2, B_ACC = B_SEMPTY + 2, B_EDONE = B_ACC + 1,
            B_MDONE = B_EDONE + 1;
  unsigned char* sZR = stgG;                    // after the mainloop of an n-block
  unsigned char* sXK = stgG + NI * GT;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * 128 * NI;
  const int nkb = wa.nkb;

  if (threadIdx.x == 0) {
    mbar_init(BAR(B_ZX), 1);
    mbar_init(BAR(B_TILE), 1);
    mbar_init(BAR(B_MDONE), 1);
    for (int s = 0; s < ST; ++s) {
      mbar_init(BAR(B_LD + s), 1);
      mbar_init(BAR(B_TEMPTY + s), 1);
    }
    for (int s = 0; s < SG; ++s) {
      mbar_init(BAR(B_GEN + s), NTW);
      mbar_init(BAR(B_GEMPTY + s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(BAR(B_SFULL + b), 1);
      mbar_init(BAR(B_SEMPTY + b), NTW);
    }
    mbar_init(BAR(B_ACC), 1);
    mbar_init(BAR(B_EDONE), NTW);
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
    int g = 0, lt = 0, nzx = 0;
    bool ok = true;
    for (int nb = blockIdx.x; nb < wa.nblk && ok; nb += gridDim.x, ++lt) {
      // the previous n-block's MMAs (readers of sXR and of the epilogue
      // exponent's operands) have completed
      if (lt > 0 && !mbar_wait(BAR(B_ACC), (lt - 1) & 1)) { ok = false; break; }
      if (*abort_flag) { ok = false; break; }
      mbar_expect_tx(BAR(B_TILE), GT);
      tma_load_2d(smem_u32(sXR), &tmXR, 0, nb * 128, BAR(B_TILE));
      for (int kb = 0; kb < nkb; ++kb, ++g) {
        const int s = g % ST;
        if (!mbar_wait(BAR(B_TEMPTY + s), ((g / ST) & 1) ^ 1) || *abort_flag) { ok = false; break; }
        unsigned char* st = stgT + s * G::TSTAGE;
        const uint32_t fb = BAR(B_LD + s);
        mbar_expect_tx(fb, CT + NI * G::NS * GT);
        tma_load_2d(smem_u32(st), &tmZK, 0, kb * KB, fb);
        for (int ib = 0; ib < NI; ++ib) {
          unsigned char* pt = st + G::OFF_P + ib * G::NS * GT;
          tma_load_2d(smem_u32(pt), &tmP, kb * KB, m0 + 128 * ib, fb);
          if (NSPLIT == 3) tma_load_2d(smem_u32(pt + GT), &tmPl, kb * KB, m0 + 128 * ib, fb);
        }
      }
      if (!ok) break;
      // the epilogue exponent's operands into the generated ring, once the
      // n-block's main MMAs (its last readers) are done
      if (!mbar_wait(BAR(B_MDONE), lt & 1) || *abort_flag) { ok = false; break; }
      mbar_expect_tx(BAR(B_ZX), (NI + 1) * GT);
      for (int ib = 0; ib < NI; ++ib) tma_load_2d(smem_u32(sZR + ib * GT), &tmZR, 0, m0 + 128 * ib, BAR(B_ZX));
      tma_load_2d(smem_u32(sXK), &tmXK, 0, nb * 128, BAR(B_ZX));
      ++nzx;
    }
    if (!ok) *abort_flag = 1;
    // every copy this thread issued lands before the CTA exits (bounded waits)
    if (nzx > 0) mbar_wait(BAR(B_ZX), (nzx - 1) & 1);
    if (lt > 0) mbar_wait(BAR(B_TILE), (lt - 1) & 1);
    if (*abort_flag) {
      for (int q = *consumed; q < g; ++q) mbar_wait(BAR(B_LD + q % ST), (q / ST) & 1);
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    // Per n-block an event-driven loop: the exponent MMA of k-block d goes out
    // as soon as its coordinates have landed and its TMEM buffer is free, ahead
    // of the main MMA of earlier k-blocks (which waits for their generated
    // tiles); then the epilogue exponents T.  Each poll tries the main MMA
    // first; the ring positions are running counters (no divisions in the
    // polling loop, whose speed shows in the launch time).
    bool ok = true;
    int g = 0, lt = 0;
    // ring positions carried across n-blocks: the exponent MMA's TMA slot,
    // the main MMA's TMA slot and its generated slot (with phases)
    int xs = 0, xph = 0, ms = 0, gsl = 0, gph = 0;
    for (int nb = blockIdx.x; nb < wa.nblk && ok; nb += gridDim.x, ++lt) {
      if (!mbar_wait(BAR(B_TILE), lt & 1)) { ok = false; break; }
      // the epilogue of the previous n-block has read the accumulators and T
      if (lt > 0 && !mbar_wait(BAR(B_EDONE), (lt - 1) & 1)) { ok = false; break; }
      fence_after();
      const uint64_t ra = sw128_desc(smem_u32(sXR));
      int d = 0, mn = 0, idle = 0;
      long long idle_since = 0;
      while (mn < nkb) {
        bool progressed = false;
        // The first main MMA of an n-block overwrites the accumulator: it waits
        // for that k-block's generated operand, which the transform warps
        // produce only after their epilogue of the previous n-block has read
        // the accumulator and the exponents T.
        if (mn < d && mbar_test(BAR(B_GEN + gsl), gph)) {
          fence_after();
          unsigned char* st = stgT + ms * G::TSTAGE;
          unsigned char* gs = stgG + gsl * G::GSTAGE;
          const uint64_t bd = sw128_desc(smem_u32(gs));
          const uint64_t bdl = sw128_desc(smem_u32(gs + GT));
#pragma unroll
          for (int ib = 0; ib < NI; ++ib) {
            const uint64_t ad = sw128_desc(smem_u32(st + G::OFF_P + ib * G::NS * GT));
            const uint64_t adl = sw128_desc(smem_u32(st + G::OFF_P + ib * G::NS * GT + GT));
#pragma unroll
            for (int kk = 0; kk < KB / 16; ++kk) {
              const uint64_t o = (uint64_t)(kk * 2);
              mma_bf16(tmem + G::ACC(ib), ad + o, bd + o, ID_MAIN, (mn | kk) != 0);
              if (NSPLIT == 3) {
                mma_bf16(tmem + G::ACC(ib), ad + o, bdl + o, ID_MAIN, 1);
                mma_bf16(tmem + G::ACC(ib), adl + o, bd + o, ID_MAIN, 1);
              }
            }
          }
          mma_commit(BAR(B_TEMPTY + ms));
          mma_commit(BAR(B_GEMPTY + gsl));
          if (++ms == ST) ms = 0;
          if (++gsl == SG) { gsl = 0; gph ^= 1; }
          ++mn;
          progressed = true;
        }
        const int gd = g + d;
        if (d < nkb && mbar_test(BAR(B_LD + xs), xph) &&
            mbar_test(BAR(B_SEMPTY + (gd & 1)), ((gd >> 1) & 1) ^ 1)) {
          fence_after();
          *consumed = gd + 1;
          const uint64_t kd = sw128_desc(smem_u32(stgT + xs * G::TSTAGE));
#pragma unroll
          for (int kk = 0; kk < KB / 16; ++kk) {
            const uint64_t o = (uint64_t)(kk * 2);
            mma_bf16(tmem + G::SB(gd & 1), ra + o, kd + o, ID_DIST, kk != 0);
          }
          mma_commit(BAR(B_SFULL + (gd & 1)));
          if (++xs == ST) { xs = 0; xph ^= 1; }
          ++d;
          progressed = true;
        }
        // the time limit and the abort flag are checked every 64 idle polls
        if (progressed) {
          idle = 0;
        } else if ((++idle & 63) == 0) {
          const long long now = clock64();
          if (idle == 64) idle_since = now;
          else if (now - idle_since > WAIT_CYCLES || *abort_flag) { ok = false; break; }
        }
      }
      g += nkb;
      if (!ok) break;
      mma_commit(BAR(B_MDONE));                  // arrives when this n-block's main MMAs are done
      if (!mbar_wait(BAR(B_ZX), lt & 1)) { ok = false; break; }
      fence_after();
      // epilogue exponents T[i, n] = log2 Kuf_in of each row block
      const uint64_t xd = sw128_desc(smem_u32(sXK));
#pragma unroll
      for (int ib = 0; ib < NI; ++ib) {
        const uint64_t zd = sw128_desc(smem_u32(sZR + ib * GT));
#pragma unroll
        for (int kk = 0; kk < KB / 16; ++kk) {
          const uint64_t o = (uint64_t)(kk * 2);
          mma_bf16(tmem + G::T(ib), zd + o, xd + o, ID_MAIN, kk != 0);
        }
      }
      mma_commit(BAR(B_ACC));
    }
    if (!ok) {
      *abort_flag = 1;
      mma_commit(BAR(B_ACC));
    }
  } else if (warp >= 2) {
    // ---------------- transform, then epilogue, per n-block ----------------
    const int quad = warp & 3, half = (warp - 2) >> 2;
    const int row = quad * 32 + lane, kcol0 = half * 32;
    const int tid = threadIdx.x - 64;                     // 0 .. 255
    const uint32_t lane_off = (uint32_t)(quad * 32) << 16;
    const int D = we.gen.D, Dp = (D + 3) & ~3, B = we.gen.B;
    const bool grad = wa.rowpart != nullptr;
    // Row sums in groups of four lanes: lane r (= lane mod 4) of a group
    // accumulates S1, S2 of the group's four rows for its DQ dimensions
    // d = r DQ + j, taking the other rows' A values by shuffles; each x~ row is
    // staged as four lane slots of DQP (>= DQ, even) floats, XW per point.
    constexpr int DQ = DP / 4, DQP = (DQ + 1) & ~1, XW = 4 * DQP;
    const int r4 = lane & 3;
    float* colbuf = ebuf;
    float* gq = ebuf + 128;
    float* xq = ebuf + 256;
    float cv[NI], cn = 0.f;
#pragma unroll
    for (int ib = 0; ib < NI; ++ib) {
      const int i = m0 + 128 * ib + row;
      cv[ib] = (grad && i < we.gen.M) ? we.c * __ldg(we.v + i) : 0.f;
    }
    if (grad && !we.hn) cn = we.c / *we.noise;          // Gaussian: -2 c h_n = c / noise
    // S0 of the thread's own row; S1p[ib][k][j] = (S1, S1) of row 4 (lane / 4)
    // + (r4 ^ k) at dimensions r4 DQ + 2j, 2j + 1 (packed FP32 pairs), likewise S2p
    float S0[NI];
    f32x2 S1p[NI][4][DQP / 2], S2p[NI][4][DQP / 2];
#pragma unroll
    for (int ib = 0; ib < NI; ++ib) {
      S0[ib] = 0.f;
#pragma unroll
      for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int j = 0; j < DQP / 2; ++j) { S1p[ib][k][j] = 0ull; S2p[ib][k][j] = 0ull; }
    }
    int g = 0, lt = 0;
    for (int nb = blockIdx.x; nb < wa.nblk; nb += gridDim.x, ++lt) {
      const int n0 = nb * 128;
      for (int kb = 0; kb < nkb; ++kb, ++g) {
        if (*abort_flag) continue;
        const int s = g % SG, b = g & 1;
        if (!mbar_wait(BAR(B_SFULL + b), (g >> 1) & 1)) { *abort_flag = 1; continue; }
        fence_after();
        float t[32];
        tmem_ld32(tmem + lane_off + G::SB(b) + kcol0, t);
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(BAR(B_SEMPTY + b));
        // generated stage s is free once the main MMA of k-block g - SG finished
        if (!mbar_wait(BAR(B_GEMPTY + s), ((g / SG) & 1) ^ 1)) { *abort_flag = 1; continue; }
        unsigned char* gs = stgG + s * G::GSTAGE;
        gen32<NSPLIT>(t, gs, gs + GT, row, kcol0);
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(BAR(B_GEN + s));
      }
      // epilogue of this n-block; its global inputs (x~ rows, g_n, h_n) are
      // fetched before the wait for the accumulators
      constexpr int PER = 128 * XW / 256;
      float xv[PER];
      float gv = 0.f, hv = 0.f;
      if (grad) {
#pragma unroll
        for (int u = 0; u < PER; ++u) {
          const int e = tid + 256 * u, n = e / XW, sl = e - n * XW, j = sl % DQP, d = (sl / DQP) * DQ + j;
          xv[u] = (n0 + n < B && j < DQ && d < D) ? __ldg(we.gen.Xs + (size_t)(n0 + n) * Dp + d) : 0.f;
        }
        if (tid < 128 && n0 + tid < B) {
          gv = __ldg(we.g + n0 + tid);
          hv = we.hn ? -2.0f * we.c * __ldg(we.hn + n0 + tid) : cn;
        }
      }
      bool ok = !*abort_flag;
      if (ok && !mbar_wait(BAR(B_ACC), lt & 1)) { *abort_flag = 1; ok = false; }
      fence_after();
      if (ok) {
        if (grad) {
#pragma unroll
          for (int u = 0; u < PER; ++u) xq[tid + 256 * u] = xv[u];
          if (tid < 128) gq[tid] = gv;
        }
        // gradient mode: colbuf holds -2 c h_n of the n-block; variance mode: the column sums
        if (tid < 128) colbuf[tid] = hv;
      }
      asm volatile("bar.sync 1, %0;" ::"n"(32 * NTW) : "memory");
      if (ok) {
        // CWD-column chunks of every row block at once (accumulator and T
        // loaded together, one wait); each x~ row read from shared memory
        // serves the four rows of a lane group and the NI row blocks
        constexpr int CWD = NI == 1 ? 16 : 8;
        for (int ch = (64 / CWD) * half; ch < (64 / CWD) * (half + 1); ++ch) {
          float w[NI][CWD], tt[NI][CWD];
          if constexpr (NI == 1) {
            tmem_ld16x2(tmem + lane_off + G::ACC(0) + (uint32_t)(ch * CWD), tmem + lane_off + G::T(0) + (uint32_t)(ch * CWD),
                        w[0], tt[0]);
          } else {
            float v4[4][8];
            const uint32_t ta[4] = {tmem + lane_off + G::ACC(0) + (uint32_t)(ch * CWD),
                                    tmem + lane_off + G::T(0) + (uint32_t)(ch * CWD),
                                    tmem + lane_off + G::ACC(1) + (uint32_t)(ch * CWD),
                                    tmem + lane_off + G::T(1) + (uint32_t)(ch * CWD)};
            tmem_ld8x4(ta, v4);
#pragma unroll
            for (int q = 0; q < CWD; ++q) {
              w[0][q] = v4[0][q]; tt[0][q] = v4[1][q];
              w[NI - 1][q] = v4[2][q]; tt[NI - 1][q] = v4[3][q];
            }
          }
          if (grad) {
#pragma unroll
            for (int q = 0; q < CWD; ++q) {
              const int n = ch * CWD + q;
              const float gn = gq[n], hn = colbuf[n];
              // the lane's slot of x~_n (a broadcast to the eight groups) and x~^2
              f32x2 xp[DQP / 2], xx[DQP / 2];
              const float* xs = xq + n * XW + r4 * DQP;
              if (DQP % 4 == 0) {
#pragma unroll
                for (int j = 0; j < DQP / 4; ++j) {
                  const ulonglong2 x = reinterpret_cast<const ulonglong2*>(xs)[j];
                  xp[2 * j] = x.x;
                  xp[2 * j + 1] = x.y;
                }
              } else {
#pragma unroll
                for (int j = 0; j < DQP / 2; ++j) xp[j] = reinterpret_cast<const f32x2*>(xs)[j];
              }
#pragma unroll
              for (int j = 0; j < DQP / 2; ++j) xx[j] = mul2(xp[j], xp[j]);
#pragma unroll
              for (int ib = 0; ib < NI; ++ib) {
                const float a = ex2(tt[ib][q]) * fmaf(cv[ib], gn, hn * w[ib][q]);
                S0[ib] += a;
                float ak[4];
                ak[0] = a;
                ak[1] = __shfl_xor_sync(0xffffffffu, a, 1);
                ak[2] = __shfl_xor_sync(0xffffffffu, a, 2);
                ak[3] = __shfl_xor_sync(0xffffffffu, a, 3);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                  const f32x2 a2 = pack2(ak[k], ak[k]);
#pragma unroll
                  for (int j = 0; j < DQP / 2; ++j) {
                    fma2(S1p[ib][k][j], a2, xp[j]);
                    fma2(S2p[ib][k][j], a2, xx[j]);
                  }
                }
              }
            }
          } else if (we.colsum) {
#pragma unroll
            for (int q = 0; q < CWD; ++q) {
              float sv = 0.f;
#pragma unroll
              for (int ib = 0; ib < NI; ++ib) sv = fmaf(ex2(tt[ib][q]), w[ib][q], sv);
#pragma unroll
              for (int o = 16; o > 0; o >>= 1) sv += __shfl_xor_sync(0xffffffffu, sv, o);
              if (lane == 0) atomicAdd(colbuf + ch * CWD + q, sv);
            }
          }
        }
      }
      fence_before();
      asm volatile("bar.sync 1, %0;" ::"n"(32 * NTW) : "memory");
      // accumulators and T of this n-block are read: the MMA warp may go on
      if (lane == 0) mbar_arrive(BAR(B_EDONE));
      if (ok && we.colsum && tid < 128 && n0 + tid < B) atomicAdd(we.colsum + n0 + tid, colbuf[tid]);
    }
    // combine the two column halves and write this CTA's partial rows
    if (grad) {
      constexpr int CW = 2 * DP + 1;
      float* comb = ebuf;                                 // colbuf, gq and xq are done with
#pragma unroll
      for (int ib = 0; ib < NI; ++ib) {
        const int i = m0 + 128 * ib + row;
        if (ib > 0) asm volatile("bar.sync 1, %0;" ::"n"(32 * NTW) : "memory");   // comb is free again
        // the two column halves' partial sums meet in comb[row][2 DP + 1]:
        // half 1 stores its values, half 0 adds its own, then the rows go out
#pragma unroll
        for (int hh = 1; hh >= 0; --hh) {
          if (half == hh) {
            if (hh == 1) comb[row * CW + 2 * DP] = S0[ib];
            else comb[row * CW + 2 * DP] += S0[ib];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              float* cr = comb + (quad * 32 + (lane & ~3) + (r4 ^ k)) * CW;
#pragma unroll
              for (int j = 0; j < DQP / 2; ++j) {
                float a1, b1, a2, b2;
                unpack2(S1p[ib][k][j], a1, b1);
                unpack2(S2p[ib][k][j], a2, b2);
                const int d0 = r4 * DQ + 2 * j;
                if (2 * j < DQ) {
                  cr[d0] = hh == 1 ? a1 : cr[d0] + a1;
                  cr[DP + d0] = hh == 1 ? a2 : cr[DP + d0] + a2;
                }
                if (2 * j + 1 < DQ) {
                  cr[d0 + 1] = hh == 1 ? b1 : cr[d0 + 1] + b1;
                  cr[DP + d0 + 1] = hh == 1 ? b2 : cr[DP + d0 + 1] + b2;
                }
              }
            }
          }
          asm volatile("bar.sync 1, %0;" ::"n"(32 * NTW) : "memory");
        }
        if (half == 0 && !*abort_flag) {
          const float s0 = comb[row * CW + 2 * DP];
          const int W = 2 * D + 1;
          float* out = wa.rowpart + (size_t)blockIdx.x * W * wa.Mp + i;
#pragma unroll
          for (int d = 0; d < DP; ++d) {
            if (d < D) {
              const float s1 = comb[row * CW + d], s2 = comb[row * CW + DP + d];
              const float z = i < we.gen.M ? __ldg(we.gen.Zs + (size_t)i * Dp + d) : 0.f;
              out[(size_t)d * wa.Mp] = fmaf(-z, s0, s1);
              out[(size_t)(D + d) * wa.Mp] = fmaf(z, fmaf(z, s0, -2.0f * s1), s2);
            }
          }
          out[(size_t)(2 * D) * wa.Mp] = s0;
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) atomicOr(wa.errword, ERRBIT_TIMEOUT);
  if (warp == 1) {
    fence_after();
    tmem_dealloc(tmem, G::TMEM_COLS);
  }
}

template <int NSPLIT, int DP, int NI>
void set_w_attr() {
  cudaFuncSetAttribute(w_tc_kernel<NSPLIT, DP, NI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       WGeo<NSPLIT, NI>::SMEM);
}

template <int NSPLIT, int NI>
void launch_w(dim3 grid, cudaStream_t st, const CUtensorMap (&m)[6], const WArgs& wa, const WEpi& we) {
  const int D = we.gen.D;
  constexpr int SM = WGeo<NSPLIT, NI>::SMEM;
  svgp_note_launch();
  if (D <= 4)
    pdl_launch(w_tc_kernel<NSPLIT, 4, NI>, grid, THREADS, SM, st, m[0], m[1], m[2], m[3], m[4], m[5], wa, we);
  else if (D <= 8)
    pdl_launch(w_tc_kernel<NSPLIT, 8, NI>, grid, THREADS, SM, st, m[0], m[1], m[2], m[3], m[4], m[5], wa, we);
  else if (D <= 16)
    pdl_launch(w_tc_kernel<NSPLIT, 16, NI>, grid, THREADS, SM, st, m[0], m[1], m[2], m[3], m[4], m[5], wa, we);
  else if constexpr (NI == 1)   // two row blocks only for D <= 16 (w_ni)
    pdl_launch(w_tc_kernel<NSPLIT, 24, NI>, grid, THREADS, SM, st, m[0], m[1], m[2], m[3], m[4], m[5], wa, we);
}

// Row blocks per CTA: two with BF16 operands when the 128-row blocks pair up
// and the (row-pair, n-block) units still give every SM a CTA (and D <= 16:
// the register-resident row sums of 24 padded dimensions would spill).
int w_ni(bool split, int Mp, int B, int D) {
  const int nblk = (B + 127) / 128;
  return (!split && D <= 16 && (Mp / 128) % 2 == 0 && (Mp / 256) * nblk >= tc_num_sms()) ? 2 : 1;
}

}  // namespace

void tc_w_init_attributes() {
  set_w_attr<1, 4, 1>();
  set_w_attr<1, 8, 1>();
  set_w_attr<1, 16, 1>();
  set_w_attr<1, 24, 1>();
  set_w_attr<1, 4, 2>();
  set_w_attr<1, 8, 2>();
  set_w_attr<1, 16, 2>();
  set_w_attr<3, 4, 1>();
  set_w_attr<3, 8, 1>();
  set_w_attr<3, 16, 1>();
  set_w_attr<3, 24, 1>();
}

int tc_w_groups(int Mp, int B, bool split, int D) {
  const int nblk = (B + 127) / 128, rb = Mp / (128 * w_ni(split, Mp, B, D));
  int gn = tc_num_sms() / rb;
  if (gn < 1) gn = 1;
  if (gn > nblk) gn = nblk;
  return gn;
}

int tc_w(const GemmCtx& g, const bf16* P, const KufTC& t, const WEpi& we, float* rowpart) {
  if (!tc_kuf_supported(we.gen.D) || we.gen.D > DPMAX) return -1;
  const int B = we.gen.B;
  const int Bp = (B + 127) / 128 * 128;
  CUtensorMap m[6];
  if (!tc_make_map(&m[0], t.ZR, g.Mp, 64, 128) || !tc_make_map(&m[1], t.ZK, g.Mp, 64, 64) ||
      !tc_make_map(&m[2], t.XR, Bp, 64, 128) || !tc_make_map(&m[3], t.XK, Bp, 64, 128) ||
      !tc_make_map(&m[4], P, g.Mp, g.Mp, 128))
    return -1;
  if (g.split) {
    if (!tc_make_map(&m[5], P + (size_t)g.Mp * g.Mp, g.Mp, g.Mp, 128)) return -1;
  } else {
    m[5] = m[4];
  }
  const int ni = w_ni(g.split, g.Mp, B, we.gen.D);
  const int gn = tc_w_groups(g.Mp, B, g.split, we.gen.D);
  WArgs wa{g.Mp / KB, Bp / 128, g.Mp, g.err, we.rowacc ? rowpart : nullptr};
  dim3 grid(gn, g.Mp / (128 * ni));
  if (g.split) launch_w<3, 1>(grid, g.st, m, wa, we);
  else if (ni == 2) launch_w<1, 2>(grid, g.st, m, wa, we);
  else launch_w<1, 1>(grid, g.st, m, wa, we);
  return wa.rowpart ? gn : 0;
}
