// tcgen05 BF16 GEMMs for sm_103a: acc[i,j] = sum_k A[i,k] B[j,k], both
// operands K-major BF16 (row-major, k contiguous), FP32 accumulation in TMEM.
//
// One 128 x 128 output tile per CTA, 192 threads:
//   warp 0      TMA producer: 128B-swizzled 128x64 tiles of A and B into a
//               STAGES-deep shared-memory ring (mbarrier full/empty pairs);
//   warp 1      TMEM allocator and MMA issuer: one elected thread issues
//               tcgen05.mma.cta_group::1.kind::f16 (M=128, N=128, K=16) x 4 per
//               k-block and frees the stage with tcgen05.commit;
//   warps 2..5  epilogue: tcgen05.ld 32x32b.x32 of their 32 TMEM lanes, then
//               the shared epilogue functors (common.cuh) write the results.
// Every mbarrier wait is bounded by a %globaltimer deadline; on expiry the
// CTA raises ERRBIT_TIMEOUT, drains its own copies and frees TMEM.
#include <cuda.h>

#include "common.cuh"
#include "internal.h"
#include "tc_common.cuh"

namespace {

constexpr int BM = 128;
constexpr int BN = 128;
constexpr int BK = 64;                      // one 128-byte swizzle atom of BF16
constexpr int TILE_BYTES = 128 * BK * 2;    // 16 KB per 128 x 64 operand tile
constexpr int EPI_SCRATCH = 4 * 32 * 33 * 4;

// Pipeline geometry per operand precision: NSPLIT = 1 (BF16) or 3 (hi/lo pairs).
template <int NSPLIT> struct Geo {
  static constexpr int NT = NSPLIT == 1 ? 2 : 4;                 // tiles per stage
  static constexpr int STAGES = NSPLIT == 1 ? 4 : 3;
  static constexpr int STAGE_BYTES = NT * TILE_BYTES;
  static constexpr int SMEM = STAGES * STAGE_BYTES + EPI_SCRATCH + 1024 + 256;
};

using namespace tc;
constexpr uint32_t IDESC = idesc_bf16(BM, BN);

// Epilogue hand-off: the warp's 32 TMEM lanes x 32 columns arrive in the row
// layout (thread = row); a padded shared-memory transpose gives the column
// layout; the functor then writes coalesced.
template <class Epi>
__device__ __forceinline__ void epi_block(Epi& epi, int i0, int j0, float (&v)[32], float* scr, int lane) {
  call_pre(epi, i0, j0, v, lane, 0);
  float vt[32];
#pragma unroll
  for (int q = 0; q < 32; ++q) scr[lane * 33 + q] = v[q];
  __syncwarp();
#pragma unroll
  for (int r = 0; r < 32; ++r) vt[r] = scr[r * 33 + lane];
  __syncwarp();
  epi.block(i0, j0, v, vt, lane);
}

template <class Epi, int NSPLIT>
__global__ void __launch_bounds__(192, 1)
tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               const __grid_constant__ CUtensorMap tmAl, const __grid_constant__ CUtensorMap tmBl,
               const Tile* __restrict__ tiles, Epi epi, int* errword) {
  using G = Geo<NSPLIT>;
  if (epi.skip()) return;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  // stage s holds tiles [A_hi, B_hi, (A_lo, B_lo)]
  float* scratch = reinterpret_cast<float*>(base + G::STAGES * G::STAGE_BYTES);
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + G::STAGES * G::STAGE_BYTES + EPI_SCRATCH);
  // bars[0..S) full, bars[S..2S) empty, bars[2S] tmem_full
  volatile uint32_t* tmem_slot = reinterpret_cast<volatile uint32_t*>(bars + 2 * G::STAGES + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + 2 * G::STAGES + 2);
  volatile int* consumed = abort_flag + 1;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const Tile tl = tiles[blockIdx.x];
  const int nk = (tl.k1 - tl.k0) / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < G::STAGES; ++s) {
      mbar_init(smem_u32(&bars[s]), 1);
      mbar_init(smem_u32(&bars[G::STAGES + s]), 1);
    }
    mbar_init(smem_u32(&bars[2 * G::STAGES]), 1);
    *abort_flag = 0;
    *consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&tmA) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&tmB) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32((const void*)tmem_slot)),
                 "r"(BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    int issued = 0;
    for (int kb = 0; kb < nk; ++kb) {
      int s = kb % G::STAGES;
      uint32_t ph = (kb / G::STAGES) & 1;
      if (!mbar_wait(smem_u32(&bars[G::STAGES + s]), ph ^ 1)) { *abort_flag = 1; break; }
      if (*abort_flag) break;
      uint32_t fb = smem_u32(&bars[s]);
      mbar_expect_tx(fb, G::STAGE_BYTES);
      int k = tl.k0 + kb * BK;
      unsigned char* st = base + s * G::STAGE_BYTES;
      tma_load_2d(smem_u32(st), &tmA, k, tl.m0, fb);
      tma_load_2d(smem_u32(st + TILE_BYTES), &tmB, k, tl.n0, fb);
      if (NSPLIT == 3) {
        tma_load_2d(smem_u32(st + 2 * TILE_BYTES), &tmAl, k, tl.m0, fb);
        tma_load_2d(smem_u32(st + 3 * TILE_BYTES), &tmBl, k, tl.n0, fb);
      }
      issued = kb + 1;
    }
    // On abort, wait (bounded) for copies that nobody consumed.
    if (*abort_flag) {
      for (int kb = *consumed; kb < issued; ++kb) mbar_wait(smem_u32(&bars[kb % G::STAGES]), (kb / G::STAGES) & 1);
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    for (int kb = 0; kb < nk; ++kb) {
      int s = kb % G::STAGES;
      uint32_t ph = (kb / G::STAGES) & 1;
      if (!mbar_wait(smem_u32(&bars[s]), ph)) { *abort_flag = 1; break; }
      fence_after();
      unsigned char* st = base + s * G::STAGE_BYTES;
      uint64_t ad = sw128_desc(smem_u32(st));
      uint64_t bd = sw128_desc(smem_u32(st + TILE_BYTES));
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) {
        mma_bf16(tmem, ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2), IDESC, (kb | kk) != 0);
        if (NSPLIT == 3) {
          uint64_t adl = sw128_desc(smem_u32(st + 2 * TILE_BYTES));
          uint64_t bdl = sw128_desc(smem_u32(st + 3 * TILE_BYTES));
          mma_bf16(tmem, ad + (uint64_t)(kk * 2), bdl + (uint64_t)(kk * 2), IDESC, 1);
          mma_bf16(tmem, adl + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2), IDESC, 1);
        }
      }
      mma_commit(smem_u32(&bars[G::STAGES + s]));
      *consumed = kb + 1;
    }
    if (nk > 0) mma_commit(smem_u32(&bars[2 * G::STAGES]));
  }
  __syncwarp();

  // ---------------- epilogue ----------------
  epi.begin_tile(tl.m0, tl.n0);
  if (warp >= 2) {
    const int quad = warp & 3;
    bool ok = true;
    if (nk > 0) {
      ok = mbar_wait(smem_u32(&bars[2 * G::STAGES]), 0);
      fence_after();
    }
    if (!ok) *abort_flag = 1;
    float* scr = scratch + (warp - 2) * 32 * 33;
    float v[32];
    for (int c = 0; c < BN / 32; ++c) {
      if (nk > 0 && ok) {
        tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(c * 32), v);
      } else {
#pragma unroll
        for (int q = 0; q < 32; ++q) v[q] = 0.f;
      }
      if (ok) epi_block(epi, tl.m0 + quad * 32, tl.n0 + c * 32, v, scr, lane);
    }
  }
  epi.reduce();
  fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) atomicOr(errword, ERRBIT_TIMEOUT);
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
  }
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
  cudaFuncSetAttribute(tc_gemm_kernel<Epi, NSPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, Geo<NSPLIT>::SMEM);
}

template <class Epi>
void set_attr_both() {
  set_attr<Epi, 1>();
  set_attr<Epi, 3>();
}

}  // namespace

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

bool tc_available() {
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  return major == 10 && minor == 3 && encode_fn() != nullptr;
}

template <class Epi>
bool tc_gemm(const GemmCtx& g, int tab, const bf16* A, const bf16* B, const Epi& e) {
  const size_t MM = (size_t)g.Mp * g.Mp;
  CUtensorMap ma, mb, mal, mbl;
  if (!tc_make_map(&ma, A, g.Mp, g.Mp, 128) || !tc_make_map(&mb, B, g.Mp, g.Mp, 128)) return false;
  if (g.split) {
    if (!tc_make_map(&mal, A + MM, g.Mp, g.Mp, 128) || !tc_make_map(&mbl, B + MM, g.Mp, g.Mp, 128)) return false;
    svgp_note_launch();
    tc_gemm_kernel<Epi, 3><<<g.nt[tab], 192, Geo<3>::SMEM, g.st>>>(ma, mb, mal, mbl, g.tt[tab], e, g.err);
  } else {
    svgp_note_launch();
    tc_gemm_kernel<Epi, 1><<<g.nt[tab], 192, Geo<1>::SMEM, g.st>>>(ma, mb, ma, mb, g.tt[tab], e, g.err);
  }
  return true;
}

#define SVGP_TC_INST(...) \
  template bool tc_gemm<__VA_ARGS__>(const GemmCtx&, int, const bf16*, const bf16*, const __VA_ARGS__&);
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

void tc_init_attributes() {
  set_attr_both<EpiVt<bf16*>>();
  set_attr_both<EpiSym<bf16*, 0>>();
  set_attr_both<EpiSym<bf16*, 1>>();
  set_attr_both<EpiSym<bf16*, 2>>();
  set_attr_both<EpiStore<bf16*>>();
  set_attr_both<EpiP<bf16*>>();
  set_attr_both<EpiVt<SplitPtr>>();
  set_attr_both<EpiSym<SplitPtr, 0>>();
  set_attr_both<EpiSym<SplitPtr, 1>>();
  set_attr_both<EpiSym<SplitPtr, 2>>();
  set_attr_both<EpiStore<SplitPtr>>();
  set_attr_both<EpiP<SplitPtr>>();
  set_attr_both<EpiLupd>();
  set_attr_both<EpiGK>();
}

