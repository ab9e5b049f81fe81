// Psi = Kuf Kuf^T (Eq. (7) data term of the bound and its gradient) with both
// SE-ARD operands generated on chip (kuf_common.cuh), so Kuf is never written
// to global memory:
//   Psi[i, j] = sum_n Kuf[i, n] Kuf[j, n]
// over the lower tile table (the epilogue mirrors).  Warp roles (320
// threads): 0 TMA producer, 1 TMEM allocator + MMA issuer, 2..9 transform and
// then epilogue (warp w covers TMEM lanes 32 (w mod 4) .. +31 and one half of
// the columns).  All waits are bounded.
//
// This file also holds the per-point preparation of the exponent-MMA operands
// shared with the W kernel (gemm_w_tc.cu).
#include "common.cuh"
#include "internal.h"
#include "kuf_common.cuh"
#include "tc_common.cuh"

namespace {

using namespace tc;
using namespace kuf;

constexpr float SQRT_LOG2E = 1.2011224087864498f;   // sqrt(log2(e))

template <int NSPLIT>
struct PsiGeo {
  static constexpr int NS = NSPLIT == 3 ? 2 : 1;                         // hi (+lo) planes
  // Two rings: the x coordinate tiles (CT each, read by the exponent MMAs, so
  // a stage frees as soon as they are done and the copies run well ahead)
  // and the generated tiles [rows I: NS*GT][rows J: NS*GT] (read by the main
  // MMAs).
  static constexpr int SC = 6;
  static constexpr int SG = NSPLIT == 3 ? 2 : 3;
  static constexpr int OFF_GA = 0;
  static constexpr int OFF_GB = NS * GT;
  static constexpr int GSTAGE = 2 * NS * GT;
  static constexpr int STATIC = 2 * GT;                                  // z rows of I and J
  static_assert(SG * GSTAGE >= NTW * 32 * 33 * 4, "epilogue scratch");
  static constexpr int NBAR = 2 * SC + 2 * SG + 6;
  static constexpr int SMEM = 1024 + STATIC + SC * CT + SG * GSTAGE + 8 * NBAR + 64;
  static_assert(SMEM <= 232448, "shared memory budget");
  static constexpr uint32_t TMEM_COLS = 512;
  // TMEM columns: accumulator [0,128); exponent buffers of 64 columns after it
  __host__ __device__ static constexpr uint32_t S_A(int b) { return 128 + 64 * b; }
  __host__ __device__ static constexpr uint32_t S_B(int b) { return 256 + 64 * b; }
};

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

template <int NSPLIT>
__global__ void __launch_bounds__(THREADS, 1)
psi_tc_kernel(const __grid_constant__ CUtensorMap tmRow,     // z, row role
              const __grid_constant__ CUtensorMap tmK,       // x, k role
              const Tile* __restrict__ tiles, int nkb, int* errword, EpiPsi epsi) {
  pdl_enter();
  using G = PsiGeo<NSPLIT>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sRowA = base;                                   // z rows of I
  unsigned char* sRowB = base + GT;                              // z rows of J
  unsigned char* cring = base + G::STATIC;                        // coordinate ring
  unsigned char* stg = cring + G::SC * CT;                        // generated ring
  uint64_t* bars = reinterpret_cast<uint64_t*>(stg + G::SG * G::GSTAGE);
  volatile uint32_t* tmem_slot = reinterpret_cast<volatile uint32_t*>(bars + G::NBAR);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* consumed = abort_flag + 1;
  constexpr int SC = G::SC, SG = G::SG;
  auto BAR = [&](int idx) { return smem_u32(&bars[idx]); };
  // LD / TEMPTY: coordinate stage landed / free; GEN / EMPTY: generated stage
  // written / free
  const int B_STATIC = 0, B_LD = 1, B_TEMPTY = 1 + SC, B_GEN = 1 + 2 * SC, B_EMPTY = 1 + 2 * SC + SG,
            B_SFULL = 1 + 2 * SC + 2 * SG, B_SEMPTY = B_SFULL + 2, B_ACC = B_SFULL + 4;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = tiles[blockIdx.x].m0, n0 = tiles[blockIdx.x].n0;
  const bool diag = m0 == n0;

  if (threadIdx.x == 0) {
    mbar_init(BAR(B_STATIC), 1);
    for (int s = 0; s < SC; ++s) {
      mbar_init(BAR(B_LD + s), 1);
      mbar_init(BAR(B_TEMPTY + s), 1);
    }
    for (int s = 0; s < SG; ++s) {
      mbar_init(BAR(B_GEN + s), NTW);
      mbar_init(BAR(B_EMPTY + s), 1);
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
    mbar_expect_tx(sb, diag ? GT : 2 * GT);
    tma_load_2d(smem_u32(sRowA), &tmRow, 0, m0, sb);
    if (!diag) tma_load_2d(smem_u32(sRowB), &tmRow, 0, n0, sb);
    int issued = 0;
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % SC;
      if (!mbar_wait(BAR(B_TEMPTY + s), ((kb / SC) & 1) ^ 1)) { *abort_flag = 1; break; }
      if (*abort_flag) break;
      const uint32_t fb = BAR(B_LD + s);
      mbar_expect_tx(fb, CT);
      tma_load_2d(smem_u32(cring + s * CT), &tmK, 0, kb * KB, fb);
      issued = kb + 1;
    }
    mbar_wait(sb, 0);
    if (*abort_flag) {
      for (int kb = *consumed; kb < issued; ++kb) mbar_wait(BAR(B_LD + kb % SC), (kb / SC) & 1);
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    // Event-driven issue: the exponent MMA of k-block d goes out as soon as its
    // coordinates have landed and its TMEM buffer is free, ahead of the main
    // MMA of earlier k-blocks, which waits for their generated tiles.  The
    // exponent MMAs therefore run up to two k-blocks ahead of the transform.
    bool ok = mbar_wait(BAR(B_STATIC), 0);
    fence_after();
    const uint64_t ra = sw128_desc(smem_u32(sRowA));
    const uint64_t rb = sw128_desc(smem_u32(sRowB));
    // ring positions: the coordinate slot of the next exponent MMA and the
    // generated slot of the next main MMA (with phases); the main MMA is
    // polled first, and the time limit and the abort flag every 64 idle polls
    int d = 0, mn = 0, cs = 0, cph = 0, gsl = 0, gph = 0, idle = 0;
    long long idle_since = 0;
    while (ok && mn < nkb) {
      bool progressed = false;
      if (mn < d && mbar_test(BAR(B_GEN + gsl), gph)) {
        fence_after();
        unsigned char* st = stg + gsl * G::GSTAGE;
        const uint64_t ad = sw128_desc(smem_u32(st + G::OFF_GA));
        const uint64_t adl = sw128_desc(smem_u32(st + G::OFF_GA + GT));
        const uint64_t bd = diag ? ad : sw128_desc(smem_u32(st + G::OFF_GB));
        const uint64_t bdl = diag ? adl : sw128_desc(smem_u32(st + G::OFF_GB + GT));
#pragma unroll
        for (int kk = 0; kk < KB / 16; ++kk) {
          const uint64_t o = (uint64_t)(kk * 2);
          mma_bf16(tmem, ad + o, bd + o, ID_MAIN, (mn | kk) != 0);
          if (NSPLIT == 3) {
            mma_bf16(tmem, ad + o, bdl + o, ID_MAIN, 1);
            mma_bf16(tmem, adl + o, bd + o, ID_MAIN, 1);
          }
        }
        mma_commit(BAR(B_EMPTY + gsl));
        if (++gsl == SG) { gsl = 0; gph ^= 1; }
        ++mn;
        progressed = true;
      }
      if (d < nkb && mbar_test(BAR(B_LD + cs), cph) &&
          mbar_test(BAR(B_SEMPTY + (d & 1)), ((d >> 1) & 1) ^ 1)) {
        fence_after();
        *consumed = d + 1;
        const int b = d & 1;
        const uint64_t kd = sw128_desc(smem_u32(cring + cs * CT));
#pragma unroll
        for (int kk = 0; kk < KB / 16; ++kk) {
          const uint64_t o = (uint64_t)(kk * 2);
          mma_bf16(tmem + G::S_A(b), ra + o, kd + o, ID_DIST, kk != 0);
          if (!diag) mma_bf16(tmem + G::S_B(b), rb + o, kd + o, ID_DIST, kk != 0);
        }
        mma_commit(BAR(B_SFULL + b));
        mma_commit(BAR(B_TEMPTY + cs));
        if (++cs == SC) { cs = 0; cph ^= 1; }
        ++d;
        progressed = true;
      }
      if (progressed) {
        idle = 0;
      } else if ((++idle & 63) == 0) {
        const long long now = clock64();
        if (idle == 64) idle_since = now;
        else if (now - idle_since > WAIT_CYCLES || *abort_flag) ok = false;
      }
    }
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
      const int s = kb % SG, b = kb & 1;
      if (!mbar_wait(BAR(B_SFULL + b), (kb >> 1) & 1)) { *abort_flag = 1; break; }
      fence_after();
      float sa[32], sbv[32];
      tmem_ld32(tmem + lane_off + G::S_A(b) + kcol0, sa);
      if (!diag) tmem_ld32(tmem + lane_off + G::S_B(b) + kcol0, sbv);
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(BAR(B_SEMPTY + b));
      // the generated buffers of stage s are free once the main MMA of kb - SG finished
      if (!mbar_wait(BAR(B_EMPTY + s), ((kb / SG) & 1) ^ 1)) { *abort_flag = 1; break; }
      unsigned char* st = stg + s * G::GSTAGE;
      gen32<NSPLIT>(sa, st + G::OFF_GA, st + G::OFF_GA + GT, row, kcol0);
      if (!diag) gen32<NSPLIT>(sbv, st + G::OFF_GB, st + G::OFF_GB + GT, row, kcol0);
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(BAR(B_GEN + s));
    }
  }
  __syncwarp();

  // ---------------- epilogue (transform warps) ----------------
  if (warp >= 2) {
    const int quad = warp & 3, half = (warp - 2) >> 2;
    bool ok = mbar_wait(BAR(B_ACC), 0);
    fence_after();
    if (!ok) *abort_flag = 1;
    if (ok && !*abort_flag) {
      const uint32_t tacc = tmem + ((uint32_t)(quad * 32) << 16);
      // the pipeline buffers are idle once the accumulator is final
      float* scr = reinterpret_cast<float*>(stg) + (warp - 2) * 32 * 33;
      for (int c = 2 * half; c < 2 * half + 2; ++c) {
        float v[32];
        tmem_ld32(tacc + (uint32_t)(c * 32), v);
        epi_block32(epsi, m0 + quad * 32, n0 + c * 32, v, scr, lane);
      }
    }
  }
  fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) atomicOr(errword, ERRBIT_TIMEOUT);
  if (warp == 1) {
    fence_after();
    tmem_dealloc(tmem, G::TMEM_COLS);
  }
}

// Operand vectors of the exponent MMA (64 BF16 per point, zero padded) for
// points p (scaled coordinates, n valid rows of npad):
//   row role R = [p'hi (D), p'hi (D), p'lo (D), c_hi, c_mid, c_lo, 1, 1, 1]
//   k role   K = [p'hi (D), p'lo (D), p'hi (D), 1, 1, 1, c'_hi, c'_mid, c'_lo]
// with p' = sqrt(log2 e) p, c = -1/2 |p'|^2 and c' = c + log2(sf2); padded
// rows get c = c' = -1e30.  R_a . K_b = t(a, b) = log2 of the SE-ARD value.
// With per-point weights hw (may be null) the k-role constant is
// c' + 1/2 log2|hw_r| (c' = -1e30 where |hw_r| < 1e-30), so that the generated
// value carries a factor sqrt|hw_r|.  R may be null (k role only).
// One point set of the preparation: rows P (n valid of npad), optional
// weights, and the row-role / k-role outputs (either may be null).
struct PrepJob {
  const float* P; int n, npad; const float* hw; bf16* R; bf16* K;
};

__global__ void kuf_prep_kernel(PrepJob j0, PrepJob j1, int nb0, int D, const float* __restrict__ sf2) {
  pdl_enter();
  // blocks [0, nb0) prepare j0, the rest j1 (one launch for both point sets);
  // one row per threadIdx.y (8 rows per block), 64 threads per row
  const bool second = (int)blockIdx.x >= nb0;
  const float* __restrict__ P = second ? j1.P : j0.P;
  const int n = second ? j1.n : j0.n, npad = second ? j1.npad : j0.npad;
  const float* __restrict__ hw = second ? j1.hw : j0.hw;
  bf16* __restrict__ R = second ? j1.R : j0.R;
  bf16* __restrict__ K = second ? j1.K : j0.K;
  __shared__ float part_sum[8][2];
  const int Dp = (D + 3) & ~3;
  const int r = ((int)blockIdx.x - (second ? nb0 : 0)) * 8 + threadIdx.y;
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
  float c_k = valid ? c_row + log2f(*sf2) : -1e30f;
  if (hw && valid) {
    const float a = fabsf(hw[r]);
    c_k = a < 1e-30f ? -1e30f : c_k + 0.5f * log2f(a);
  }
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
  if (R) R[(size_t)r * 64 + d] = rv;
  K[(size_t)r * 64 + d] = kv;
}

template <int NSPLIT>
void set_psi_attr() {
  cudaFuncSetAttribute(psi_tc_kernel<NSPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, PsiGeo<NSPLIT>::SMEM);
}

}  // namespace

void k_kuf_prep(const float* Zs, const float* Xs, int M, int Mp, int B, int Bp, int D, const float* sf2,
                const KufTC& t, cudaStream_t st) {
  dim3 blk(64, 8);
  const PrepJob z{Zs, M, Mp, nullptr, t.ZR, t.ZK}, x{Xs, B, Bp, nullptr, t.XR, t.XK};
  const int nbz = (Mp + 7) / 8, nbx = (Xs && B > 0) ? (Bp + 7) / 8 : 0;
  svgp_note_launch();
  pdl_launch(kuf_prep_kernel, nbz + nbx, blk, 0, st, z, x, nbz, D, sf2);
}

void k_kuf_prep_weighted(const float* Xs, int B, int Bp, int D, const float* sf2, const float* h, bf16* XKh,
                         cudaStream_t st) {
  dim3 blk(64, 8);
  const PrepJob x{Xs, B, Bp, h, nullptr, XKh};
  svgp_note_launch();
  pdl_launch(kuf_prep_kernel, (Bp + 7) / 8, blk, 0, st, x, x, (Bp + 7) / 8, D, sf2);
}

void tc_kuf_init_attributes() {
  set_psi_attr<1>();
  set_psi_attr<3>();
  tc_w_init_attributes();
  tc_gemv_init_attributes();
}

bool tc_kuf_supported(int D) { return D >= 1 && 3 * D + 6 <= 64 && tc_available(); }

bool tc_psi(const GemmCtx& g, const KufGen& kg, const KufTC& t, const bf16* Kk, int B, EpiPsi e) {
  if (!tc_kuf_supported(kg.D)) return false;
  const int Bp = (B + 127) / 128 * 128;
  CUtensorMap mr, mk;
  if (!tc_make_map(&mr, t.ZR, g.Mp, 64, 128) || !tc_make_map(&mk, Kk, Bp, 64, 64)) return false;
  svgp_note_launch();
  if (g.split)
    pdl_launch(psi_tc_kernel<3>, g.nt[TT_PSI], THREADS, PsiGeo<3>::SMEM, g.st, mr, mk, g.tt[TT_PSI], Bp / KB, g.err, e);
  else
    pdl_launch(psi_tc_kernel<1>, g.nt[TT_PSI], THREADS, PsiGeo<1>::SMEM, g.st, mr, mk, g.tt[TT_PSI], Bp / KB, g.err, e);
  return true;
}
