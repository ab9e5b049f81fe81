// tcgen05 BF16 GEMMs for sm_103a: acc[i,j] = sum_k A[i,k] B[j,k], both
// operands K-major BF16 (row-major, k contiguous), FP32 accumulation in TMEM.
//
// Persistent kernel: one CTA per SM walks its list of 128 x 128 output tiles
// (a longest-processing-time-first schedule built on the host).  192 threads:
//   warp 0      TMA producer: 128B-swizzled 128x64 tiles of A and B (and of
//               their lo parts for split operands) into a STAGES-deep
//               shared-memory ring (mbarrier full/empty pairs) that runs
//               continuously across tiles;
//   warp 1      TMEM allocator and MMA issuer: one thread issues
//               tcgen05.mma.cta_group::1.kind::f16 (M=128, N=128, K=16) into
//               one of two TMEM accumulators (256 columns), frees stages with
//               tcgen05.commit and signals the finished accumulator;
//   warps 2..5  epilogue: tcgen05.ld 32x32b.x32 of their 32 TMEM lanes, then
//               per 32 x 32 block the functor's epilogue (epi_tc.cuh): input
//               blocks by TMA loads issued ahead, results staged in swizzled
//               shared memory and written by TMA stores; then release the
//               accumulator -- so the epilogue of tile t overlaps the
//               mainloop of tile t+1.
// Every mbarrier wait is bounded; on expiry the CTA raises ERRBIT_TIMEOUT,
// stops issuing, drains its own copies and frees TMEM.
#include <cuda.h>

#include <cstring>

#include <type_traits>

#include "common.cuh"
#include "epi_tc.cuh"
#include "internal.h"
#include "tc_common.cuh"

namespace {

constexpr int BM = 128;
constexpr int BN = 128;
constexpr int BK = 64;                      // one 128-byte swizzle atom of BF16
constexpr int TILE_BYTES = 128 * BK * 2;    // 16 KB per 128 x 64 operand tile
constexpr uint32_t TMEM_COLS = 2 * BN;      // two accumulators

// Pipeline geometry per epilogue and operand precision (NSPLIT = 1: BF16,
// 3: hi/lo pairs, 5: hi/lo A with hi/lo/lo2 B).  The mainloop streams operand tiles from L2 and its rate
// is set by the bytes in flight, so the ring takes every stage that fits
// beside the epilogue's own buffers (input slots only where the epilogue
// reads a matrix, and its staging slots).  An epilogue that reads input
// blocks keeps two slots per warp (the next block's copy in flight during the
// current block) unless the ring would have only two stages and one slot
// gives it a third: with split operands (64 KB stages) the L^T K~ product
// then runs 5 % faster (two stages leave the copies waiting for the MMAs).
template <class Epi, int NSPLIT> struct Geo {
  static constexpr int NT = NSPLIT == 1 ? 2 : NSPLIT == 3 ? 4 : 5;   // operand tiles per stage
  static constexpr int STAGE_BYTES = NT * TILE_BYTES;
  static constexpr int epi_bytes(int nin) {
    return 4 * ((etc::EpiSmem<Epi>::input ? nin * etc::SLOT : 0) + etc::EpiSmem<Epi>::out_slots * etc::SLOT);
  }
  static constexpr int fits(int st, int nin) { return st * STAGE_BYTES + epi_bytes(nin) + 1024 + 8 * (2 * st + 12) + 64 <= 232448; }
  static constexpr int stages(int nin) {
    return fits(6, nin) ? 6 : fits(5, nin) ? 5 : fits(4, nin) ? 4 : fits(3, nin) ? 3 : 2;
  }
  static constexpr int NIN = (stages(2) == 2 && stages(1) > 2) ? 1 : 2;   // input slots per epilogue warp
  static constexpr int IN = etc::EpiSmem<Epi>::input ? NIN * etc::SLOT : 0;
  static constexpr int WARP = IN + etc::EpiSmem<Epi>::out_slots * etc::SLOT;
  static constexpr int EPI_BYTES = 4 * WARP;                     // four epilogue warps
  static constexpr int fixed(int st) { return EPI_BYTES + 1024 + 8 * (2 * st + 12) + 64; }
  static constexpr int STAGES = stages(NIN);
  // [0,S) full, [S,2S) empty, acc_full[2], acc_empty[2], epilogue input[4 warps][2]
  static constexpr int NBAR = 2 * STAGES + 4 + 8;
  static constexpr int SMEM = STAGES * STAGE_BYTES + fixed(STAGES);
  static_assert(SMEM <= 232448, "shared memory budget");
};

using namespace tc;
constexpr uint32_t IDESC = idesc_bf16(BM, BN);

template <class Epi, int NSPLIT>
__global__ void __launch_bounds__(192, 1)
tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               const __grid_constant__ CUtensorMap tmAl, const __grid_constant__ CUtensorMap tmBl,
               const __grid_constant__ CUtensorMap tmBl2, const TcTile* __restrict__ tiles, const int* __restrict__ toff, Epi epi, int* errword,
               const __grid_constant__ etc::EpiMaps maps, float* __restrict__ kpart, int* kflag) {
  using G = Geo<Epi, NSPLIT>;
  constexpr int S = G::STAGES;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  // stage s holds tiles [A_hi, B_hi, (A_lo, B_lo, (B_lo2))]
  unsigned char* epi_base = base + S * G::STAGE_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(epi_base + G::EPI_BYTES);
  // bars: [0,S) full, [S,2S) empty, 2S+b acc_full[b], 2S+2+b acc_empty[b], 2S+4+2w+k epilogue input
  volatile uint32_t* tmem_slot = reinterpret_cast<volatile uint32_t*>(bars + G::NBAR);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* consumed = abort_flag + 1;
  auto BAR = [&](int i) { return smem_u32(&bars[i]); };

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  // Set-up that touches no global memory (barriers, TMEM, the tensor maps in
  // the parameter space) runs before the wait for the previous kernel, so it
  // overlaps that kernel's tail.  The TMEM allocation can only wait for a
  // co-resident CTA of an earlier kernel to free its columns, and such a CTA
  // never waits on this kernel.
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(BAR(s), 1);
      mbar_init(BAR(S + s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(BAR(2 * S + b), 1);       // acc_full: one tcgen05.commit (or arrive)
      mbar_init(BAR(2 * S + 2 + b), 4);   // acc_empty: one arrive per epilogue warp
    }
    for (int k = 0; k < 8; ++k) mbar_init(BAR(2 * S + 4 + k), 1);
    *abort_flag = 0;
    *consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&tmA) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&tmB) : "memory");
  }
  if (warp == 1) tmem_alloc(smem_u32((const void*)tmem_slot), TMEM_COLS);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  pdl_enter();
  if (epi.skip()) {
    if (warp == 1) tmem_dealloc(tmem, TMEM_COLS);
    return;
  }
  const int t_beg = toff[blockIdx.x], t_end = toff[blockIdx.x + 1];   // this CTA's tiles

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    int g = 0;          // running k-block counter over all tiles of this CTA
    for (int t = t_beg; t < t_end && !*abort_flag; ++t) {
      const TcTile tl = tiles[t];
      const int nk = (tl.k1 - tl.k0) / BK;
      for (int kb = 0; kb < nk; ++kb, ++g) {
        const int s = g % S;
        if (!mbar_wait(BAR(S + s), ((g / S) & 1) ^ 1)) { *abort_flag = 1; break; }
        if (*abort_flag) break;
        const uint32_t fb = BAR(s);
        mbar_expect_tx(fb, G::STAGE_BYTES);
        const int k = tl.k0 + kb * BK;
        unsigned char* st = base + s * G::STAGE_BYTES;
        tma_load_2d(smem_u32(st), &tmA, k, tl.m0, fb);
        tma_load_2d(smem_u32(st + TILE_BYTES), &tmB, k, tl.n0, fb);
        if (NSPLIT >= 3) {
          tma_load_2d(smem_u32(st + 2 * TILE_BYTES), &tmAl, k, tl.m0, fb);
          tma_load_2d(smem_u32(st + 3 * TILE_BYTES), &tmBl, k, tl.n0, fb);
        }
        if (NSPLIT == 5) tma_load_2d(smem_u32(st + 4 * TILE_BYTES), &tmBl2, k, tl.n0, fb);
      }
    }
    // On abort, wait (bounded) for copies that nobody consumed.
    if (*abort_flag) {
      for (int q = *consumed; q < g; ++q) mbar_wait(BAR(q % S), (q / S) & 1);
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    int g = 0, lt = 0;
    for (int t = t_beg; t < t_end; ++t, ++lt) {
      const TcTile tl = tiles[t];
      const int nk = (tl.k1 - tl.k0) / BK;
      const int b = lt & 1;
      if (!mbar_wait(BAR(2 * S + 2 + b), ((lt >> 1) & 1) ^ 1)) { *abort_flag = 1; break; }
      fence_after();
      const uint32_t acc = tmem + (uint32_t)(b * BN);
      bool ok = true;
      for (int kb = 0; kb < nk; ++kb, ++g) {
        const int s = g % S;
        if (!mbar_wait(BAR(s), (g / S) & 1)) { ok = false; break; }
        fence_after();
        unsigned char* st = base + s * G::STAGE_BYTES;
        const uint64_t ad = sw128_desc(smem_u32(st));
        const uint64_t bd = sw128_desc(smem_u32(st + TILE_BYTES));
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
          const uint64_t o = (uint64_t)(kk * 2);
          mma_bf16(acc, ad + o, bd + o, IDESC, (kb | kk) != 0);
          if (NSPLIT >= 3) {
            const uint64_t adl = sw128_desc(smem_u32(st + 2 * TILE_BYTES));
            const uint64_t bdl = sw128_desc(smem_u32(st + 3 * TILE_BYTES));
            mma_bf16(acc, ad + o, bdl + o, IDESC, 1);
            mma_bf16(acc, adl + o, bd + o, IDESC, 1);
            if (NSPLIT == 5) {
              // A_hi B_lo2 + A_lo B_lo: B to about 2^-26, A to about 2^-17
              const uint64_t bdl2 = sw128_desc(smem_u32(st + 4 * TILE_BYTES));
              mma_bf16(acc, ad + o, bdl2 + o, IDESC, 1);
              mma_bf16(acc, adl + o, bdl + o, IDESC, 1);
            }
          }
        }
        mma_commit(BAR(S + s));
        *consumed = g + 1;
      }
      if (!ok) { *abort_flag = 1; mma_commit(BAR(2 * S + b)); break; }
      if (nk > 0) mma_commit(BAR(2 * S + b));
      else mbar_arrive(BAR(2 * S + b));
      if (*abort_flag) break;
    }
  } else if (warp >= 2) {
    // ---------------- epilogue ----------------
    const int quad = warp & 3, ew = warp - 2;
    unsigned char* ein = epi_base + ew * G::WARP;              // NIN input slots (if any)
    unsigned char* eout = ein + G::IN;                         // staging slots
    const uint32_t inbar0 = BAR(2 * S + 4 + 2 * ew);
    int n_issued[2] = {0, 0}, n_used[2] = {0, 0};
    // input block of (i0, j0) into slot k (lane 0 issues; the slot's previous
    // contents were read by this warp before the preceding __syncwarp)
    auto issue_in = [&](int k, int i0, int j0) {
      int x, y;
      if (!etc::tc_in(epi, i0, j0, x, y) || etc::tc_skip(epi, i0, j0)) return;
      if (lane == 0) {
        fence_proxy_async();
        mbar_expect_tx(inbar0 + 8 * k, etc::SLOT);
        tma_load_2d(smem_u32(ein + k * etc::SLOT), &maps.in, x, y, inbar0 + 8 * k);
      }
      ++n_issued[k];
    };
    epi.begin_tile(0, 0);
    int lt = 0;
    for (int t = t_beg; t < t_end; ++t, ++lt) {
      const TcTile tl = tiles[t];
      const int nk = (tl.k1 - tl.k0) / BK;
      const int b = lt & 1;
      const int i0 = tl.m0 + quad * 32;
      const uint32_t acc = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(b * BN);
      if (tl.role == TC_PRODUCER) {
        // producer chunk of a split tile: raw FP32 partial sums of its K range
        // into the workspace slot (rows i0 .. i0 + 31), then count this warp done
        if (!mbar_wait(BAR(2 * S + b), (lt >> 1) & 1)) { *abort_flag = 1; break; }
        fence_after();
        float* dst = kpart + (size_t)tl.slot * (BM * BN) + (size_t)(quad * 32 + lane) * BN;
#pragma unroll
        for (int c = 0; c < BN / 32; ++c) {
          float v[32];
          tmem_ld32(acc + (uint32_t)(c * 32), v);
#pragma unroll
          for (int q = 0; q < 8; ++q)
            __stcg(reinterpret_cast<float4*>(dst + c * 32) + q, make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]));
        }
        fence_before();
        __threadfence();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(BAR(2 * S + 2 + b));
          atomicAdd(kflag + 2 * tl.slot, 1);
        }
        continue;
      }
      const float* part = nullptr;     // owner chunk: the producer's partial rows
      if (tl.role == TC_OWNER) part = kpart + (size_t)tl.slot * (BM * BN) + (size_t)(quad * 32 + lane) * BN;
#pragma unroll
      for (int k = 0; k < G::NIN; ++k) issue_in(k, i0, tl.n0 + 32 * k);
      etc::tc_prefetch(epi, tl.m0, tl.n0, lane);
      if (!mbar_wait(BAR(2 * S + b), (lt >> 1) & 1)) { *abort_flag = 1; break; }
      fence_after();
      if (*abort_flag) break;
      bool ok = true;
      if (part) {
        // the four producer warps of this tile have stored their partials
        // (bounded wait; the producer chunk never waits on anything)
        if (lane == 0) {
          const long long t0 = clock64();
          while (ld_acquire(kflag + 2 * tl.slot) < 4) {
            if (clock64() - t0 > WAIT_CYCLES || *abort_flag) { ok = false; break; }
            __nanosleep(64);
          }
        }
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        if (ok) (void)ld_acquire(kflag + 2 * tl.slot);
        __syncwarp();
      }
#pragma unroll
      for (int c = 0; c < BN / 32; ++c) {
        const int j0 = tl.n0 + c * 32, k = c % G::NIN;
        if (!etc::tc_skip(epi, i0, j0)) {
          float v[32];
          if (nk > 0) {
            tmem_ld32(acc + (uint32_t)(c * 32), v);
          } else {
#pragma unroll
            for (int q = 0; q < 32; ++q) v[q] = 0.f;
          }
          if (part && ok) {
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const float4 p = __ldcg(reinterpret_cast<const float4*>(part + c * 32) + q);
              v[4 * q] += p.x; v[4 * q + 1] += p.y; v[4 * q + 2] += p.z; v[4 * q + 3] += p.w;
            }
          }
          int x, y;
          if (etc::tc_in(epi, i0, j0, x, y)) {
            if (!mbar_wait(inbar0 + 8 * k, n_used[k] & 1)) { ok = false; }
            ++n_used[k];
          }
          if (lane == 0) etc::bulk_wait_read();                 // staging slots free again
          __syncwarp();
          if (ok) etc::tc_epi(epi, i0, j0, v, lane, ein + k * etc::SLOT, eout, maps);
        }
        __syncwarp();
        if (c + G::NIN < BN / 32) issue_in(k, i0, tl.n0 + (c + G::NIN) * 32);
      }
      if (!ok) *abort_flag = 1;
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(BAR(2 * S + 2 + b));
      // the last of the four owner warps to finish reading resets the slot's
      // counts for the next launch
      if (part && ok && lane == 0 && atomicAdd(kflag + 2 * tl.slot + 1, 1) == 3) {
        kflag[2 * tl.slot] = 0;
        kflag[2 * tl.slot + 1] = 0;
      }
      if (!ok) break;
    }
    // every input copy landed and every store completed before the CTA exits
    for (int k = 0; k < 2; ++k)
      for (; n_used[k] < n_issued[k]; ++n_used[k]) mbar_wait(inbar0 + 8 * k, n_used[k] & 1);
    if (lane == 0) etc::bulk_wait_all();
  }
  __syncwarp();
  if (warp < 2) epi.begin_tile(0, 0);     // zero partials of the non-epilogue warps
  epi.reduce();
  fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) atomicOr(errword, ERRBIT_TIMEOUT);
  if (warp == 1) {
    fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

// Failure-path probe: one thread waits, with the bounded wait every pipeline
// uses, on an mbarrier that nothing ever arrives on, so the wait gives up
// after `limit` cycles and raises ERRBIT_TIMEOUT as an expired pipeline
// wait does.  No copy, MMA or TMEM allocation is involved.
__global__ void wait_probe_kernel(int* errword, long long limit) {
  pdl_enter();
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(smem_u32(&bar), 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  if (!mbar_wait_for(smem_u32(&bar), 0, limit)) atomicOr(errword, ERRBIT_TIMEOUT);
}

// ---------------------------------------------------------------------------
// Host side: tensor maps and launches.
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

template <class Epi, int NSPLIT>
void set_attr() {
  cudaFuncSetAttribute(tc_gemm_kernel<Epi, NSPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, Geo<Epi, NSPLIT>::SMEM);
}

template <class Epi>
void set_attr_both() {
  set_attr<Epi, 1>();
  set_attr<Epi, 3>();
}

}  // namespace

int tc_num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 148;
  }
  return n;
}

// 2-D BF16 row-major [rows][cols] (ld = cols), box 64 (k) x box_rows (rows).
bool tc_make_map(CUtensorMap* m, const void* ptr, int rows, int cols, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

namespace {

// 32 x 32 blocks of an Mp x Mp matrix for the epilogue: FP32 with 128-byte
// rows (128-byte swizzle) or BF16 with 64-byte rows (64-byte swizzle).
bool block_map(CUtensorMap* m, const void* ptr, int Mp, bool f32) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || !ptr) return false;
  const int es = f32 ? 4 : 2;
  cuuint64_t dims[2] = {(cuuint64_t)Mp, (cuuint64_t)Mp};
  cuuint64_t strides[1] = {(cuuint64_t)Mp * es};
  cuuint32_t box[2] = {32, 32};
  cuuint32_t el[2] = {1, 1};
  CUresult r = fn(m, f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                  const_cast<void*>(ptr), dims, strides, box, el, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  f32 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}
bool out_maps(CUtensorMap* m, bf16* p, int Mp) { return block_map(m, p, Mp, false); }
bool out_maps(CUtensorMap* m, const SplitPtr& p, int Mp) {
  return block_map(m, p.hi, Mp, false) && block_map(m + 1, p.lo, Mp, false);
}

// Tensor maps of each epilogue: input block source and output planes in the
// order epi_tc.cuh stores them.  All matrices are Mp x Mp (leading dimension Mp).
template <class OutP>
bool epi_maps(const EpiVt<OutP>& e, etc::EpiMaps& m, int Mp) {
  return e.ld == Mp && (!e.s || block_map(&m.in, e.Lf, Mp, true)) && out_maps(m.out, e.out, Mp);
}
template <class OutP, int MODE>
bool epi_maps(const EpiSym<OutP, MODE>& e, etc::EpiMaps& m, int Mp) {
  return e.ld == Mp && out_maps(m.out, e.out, Mp);
}
bool epi_maps(const EpiLupd& e, etc::EpiMaps& m, int Mp) {
  return e.ld == Mp && block_map(&m.in, e.Lf, Mp, true) && block_map(&m.out[0], e.Lf, Mp, true);
}
template <class OutP>
bool epi_maps(const EpiStore<OutP>& e, etc::EpiMaps& m, int Mp) {
  return e.ld == Mp && out_maps(m.out, e.out, Mp);
}
template <class OutP>
bool epi_maps(const EpiStoreT<OutP>& e, etc::EpiMaps& m, int Mp) {
  return e.ld == Mp && out_maps(m.out, e.out, Mp);
}
template <class OutP>
bool epi_maps(const EpiP<OutP>& e, etc::EpiMaps& m, int Mp) {
  return e.ld == Mp && (!e.Psi || block_map(&m.in, e.Psi, Mp, true)) && block_map(&m.out[0], e.Pf, Mp, true) &&
         out_maps(m.out + 1, e.Plo, Mp);
}
bool epi_maps(const EpiGK& e, etc::EpiMaps& m, int Mp) {
  return e.ld == Mp && block_map(&m.in, e.Pf, Mp, true) && block_map(&m.out[0], e.GKuu, Mp, true);
}

}  // namespace

void tc_wait_probe(int* errword, cudaStream_t st) {
  svgp_note_launch();
  pdl_launch(wait_probe_kernel, 1, 32, 0, st, errword, 1ll << 26);   // about 32 ms at 2 GHz
}

bool tc_available() {
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  return major == 10 && minor == 3 && encode_fn() != nullptr;
}

template <class Epi>
bool tc_gemm(const GemmCtx& g, int tab, const bf16* A, const bf16* B, const Epi& e, const bf16* B3) {
  const size_t MM = (size_t)g.Mp * g.Mp;
  const int grid = g.ncta[tab];
  CUtensorMap ma, mb, mal, mbl, mbl2;
  if (!tc_make_map(&ma, A, g.Mp, g.Mp, 128) || !tc_make_map(&mb, B, g.Mp, g.Mp, 128)) return false;
  etc::EpiMaps em;
  memset(&em, 0, sizeof(em));
  if (!epi_maps(e, em, g.Mp)) return false;
  if (g.split && B3) {
    // B's third plane B3 (B + 2 Mp^2): only the L^T K~ product takes it
    if constexpr (std::is_same<Epi, EpiVt<SplitPtr>>::value) {
      if (B3 != B + 2 * MM) return false;
      if (!tc_make_map(&mal, A + MM, g.Mp, g.Mp, 128) || !tc_make_map(&mbl, B + MM, g.Mp, g.Mp, 128) ||
          !tc_make_map(&mbl2, B3, g.Mp, g.Mp, 128))
        return false;
      svgp_note_launch();
      pdl_launch(tc_gemm_kernel<Epi, 5>, grid, 192, Geo<Epi, 5>::SMEM, g.st, ma, mb, mal, mbl, mbl2, g.tct[tab], g.toff[tab], e,
                 g.err, em, g.kpart, g.kflag);
    } else {
      return false;
    }
  } else if (g.split) {
    if (!tc_make_map(&mal, A + MM, g.Mp, g.Mp, 128) || !tc_make_map(&mbl, B + MM, g.Mp, g.Mp, 128)) return false;
    svgp_note_launch();
    pdl_launch(tc_gemm_kernel<Epi, 3>, grid, 192, Geo<Epi, 3>::SMEM, g.st, ma, mb, mal, mbl, mbl, g.tct[tab], g.toff[tab], e, g.err,
               em, g.kpart, g.kflag);
  } else {
    svgp_note_launch();
    pdl_launch(tc_gemm_kernel<Epi, 1>, grid, 192, Geo<Epi, 1>::SMEM, g.st, ma, mb, ma, mb, mb, g.tct[tab], g.toff[tab], e, g.err,
               em, g.kpart, g.kflag);
  }
  return true;
}

#define SVGP_TC_INST(...) \
  template bool tc_gemm<__VA_ARGS__>(const GemmCtx&, int, const bf16*, const bf16*, const __VA_ARGS__&, const bf16*);
SVGP_TC_INST(EpiVt<bf16*>)
SVGP_TC_INST(EpiSym<bf16*, 0>)
SVGP_TC_INST(EpiSym<bf16*, 1>)
SVGP_TC_INST(EpiSym<bf16*, 2>)
SVGP_TC_INST(EpiStore<bf16*>)
SVGP_TC_INST(EpiP<bf16*>)
SVGP_TC_INST(EpiVt<SplitPtr>)
SVGP_TC_INST(EpiSym<SplitPtr, 0>)
SVGP_TC_INST(EpiSym<SplitPtr, 1>)
SVGP_TC_INST(EpiSym<SplitPtr, 2>)
SVGP_TC_INST(EpiStore<SplitPtr>)
SVGP_TC_INST(EpiP<SplitPtr>)
SVGP_TC_INST(EpiLupd)
SVGP_TC_INST(EpiGK)
SVGP_TC_INST(EpiStoreT<bf16*>)
SVGP_TC_INST(EpiStoreT<SplitPtr>)

void tc_init_attributes() {
  set_attr_both<EpiVt<bf16*>>();
  set_attr_both<EpiSym<bf16*, 0>>();
  set_attr_both<EpiSym<bf16*, 1>>();
  set_attr_both<EpiSym<bf16*, 2>>();
  set_attr_both<EpiStore<bf16*>>();
  set_attr_both<EpiP<bf16*>>();
  set_attr_both<EpiVt<SplitPtr>>();
  set_attr<EpiVt<SplitPtr>, 5>();
  set_attr_both<EpiSym<SplitPtr, 0>>();
  set_attr_both<EpiSym<SplitPtr, 1>>();
  set_attr_both<EpiSym<SplitPtr, 2>>();
  set_attr_both<EpiStore<SplitPtr>>();
  set_attr_both<EpiP<SplitPtr>>();
  set_attr_both<EpiLupd>();
  set_attr_both<EpiGK>();
  set_attr_both<EpiStoreT<bf16*>>();
  set_attr_both<EpiStoreT<SplitPtr>>();
}
