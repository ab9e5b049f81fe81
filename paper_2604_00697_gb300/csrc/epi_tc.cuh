// Epilogues of the tcgen05 GEMM (gemm_tc.cu) through shared memory and TMA.
//
// An epilogue warp owns 32 accumulator rows (its TMEM lane quarter) and
// handles one 32 x 32 block at a time in the row layout (thread = row i,
// v[q] = acc(i, j0 + q)):
//   * an input block of an FP32 matrix (Psi, P or L, direct or transposed)
//     arrives by a TMA tile load issued one or two blocks ahead into a
//     double-buffered 4 KB slot (128-byte swizzle);
//   * results are written into 4 KB staging slots in the TMA swizzle
//     layouts (FP32: 128-byte rows, 128-byte swizzle; BF16: 64-byte rows,
//     64-byte swizzle) -- rows by 16-byte vector stores, mirrored (transposed)
//     blocks by scalar column stores, both free of bank conflicts -- and
//     leave by TMA tile stores (bulk groups), so no global store is issued
//     per element.
// Symmetric results keep the tile-region rule of the shared functors
// (common.cuh): the computed triangle is written directly and mirrored; a
// diagonal block is assembled whole (row writes, then the mirrored entries
// over the other triangle) and stored once.
#pragma once
#include <cuda.h>

#include "common.cuh"
#include "tc_common.cuh"

namespace etc {

using namespace tc;

constexpr int SLOT = 4096;                    // one 32 x 32 FP32 block (or two BF16 blocks)
constexpr int IN_BYTES = 2 * SLOT;            // double-buffered input block

// Shared memory an epilogue needs per warp: whether it reads an input block
// (double-buffered IN_BYTES) and how many 4 KB staging slots it writes.
template <class Epi> struct EpiSmem;
template <class OutP> struct EpiSmem<EpiVt<OutP>> { static constexpr bool input = true; static constexpr int out_slots = 1; };
template <class OutP, int MODE> struct EpiSmem<EpiSym<OutP, MODE>> {
  static constexpr bool input = false; static constexpr int out_slots = 2;
};
template <> struct EpiSmem<EpiLupd> { static constexpr bool input = true; static constexpr int out_slots = 1; };
template <class OutP> struct EpiSmem<EpiStore<OutP>> { static constexpr bool input = false; static constexpr int out_slots = 1; };
template <class OutP> struct EpiSmem<EpiStoreT<OutP>> { static constexpr bool input = false; static constexpr int out_slots = 1; };
template <class OutP> struct EpiSmem<EpiP<OutP>> { static constexpr bool input = true; static constexpr int out_slots = 4; };
template <> struct EpiSmem<EpiGK> { static constexpr bool input = true; static constexpr int out_slots = 2; };

struct alignas(64) EpiMaps {
  CUtensorMap in;
  CUtensorMap out[6];
};

// ---- swizzled staging layouts ----
__device__ __forceinline__ uint32_t off32(int r, int c) {
  return (uint32_t)(r * 128 + ((((c >> 2) ^ r) & 7) << 4) + ((c & 3) << 2));
}
__device__ __forceinline__ uint32_t off16(int r, int c) {
  return (uint32_t)(r * 64 + ((((c >> 3) ^ (r >> 1)) & 3) << 4) + ((c & 7) << 1));
}

__device__ __forceinline__ uint32_t pk(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

__device__ __forceinline__ void row_f32(unsigned char* b, int r, const float (&x)[32]) {
#pragma unroll
  for (int k = 0; k < 8; ++k)
    *reinterpret_cast<float4*>(b + r * 128 + (((k ^ r) & 7) << 4)) =
        make_float4(x[4 * k], x[4 * k + 1], x[4 * k + 2], x[4 * k + 3]);
}
__device__ __forceinline__ void row_b16(unsigned char* b, int r, const float (&x)[32]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    uint4 u;
    u.x = pk(x[8 * k], x[8 * k + 1]);
    u.y = pk(x[8 * k + 2], x[8 * k + 3]);
    u.z = pk(x[8 * k + 4], x[8 * k + 5]);
    u.w = pk(x[8 * k + 6], x[8 * k + 7]);
    *reinterpret_cast<uint4*>(b + r * 64 + (((k ^ (r >> 1)) & 3) << 4)) = u;
  }
}
__device__ __forceinline__ void ld_row_f32(const unsigned char* b, int r, float (&x)[32]) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float4 f = *reinterpret_cast<const float4*>(b + r * 128 + (((k ^ r) & 7) << 4));
    x[4 * k] = f.x; x[4 * k + 1] = f.y; x[4 * k + 2] = f.z; x[4 * k + 3] = f.w;
  }
}
// x[q] = element (q, c) of an FP32 block (column c)
__device__ __forceinline__ void ld_col_f32(const unsigned char* b, int c, float (&x)[32]) {
#pragma unroll
  for (int q = 0; q < 32; ++q) x[q] = *reinterpret_cast<const float*>(b + off32(q, c));
}

// Output precision of an operand copy: one BF16 block, or BF16 hi + lo blocks
// (lo = x - hi) sharing one slot.
template <class OutP> struct Out;
template <> struct Out<bf16*> {
  static constexpr int NMAP = 1;
  __device__ static void row(unsigned char* b, int r, const float (&x)[32]) { row_b16(b, r, x); }
  __device__ static void elem(unsigned char* b, int r, int c, float x) {
    *reinterpret_cast<bf16*>(b + off16(r, c)) = __float2bfloat16_rn(x);
  }
};
template <> struct Out<SplitPtr> {
  static constexpr int NMAP = 2;
  __device__ static void row(unsigned char* b, int r, const float (&x)[32]) {
    float lo[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) lo[q] = x[q] - __bfloat162float(__float2bfloat16_rn(x[q]));
    row_b16(b, r, x);
    row_b16(b + 2048, r, lo);
  }
  __device__ static void elem(unsigned char* b, int r, int c, float x) {
    const bf16 h = __float2bfloat16_rn(x);
    *reinterpret_cast<bf16*>(b + off16(r, c)) = h;
    *reinterpret_cast<bf16*>(b + 2048 + off16(r, c)) = __float2bfloat16_rn(x - __bfloat162float(h));
  }
};
__device__ __forceinline__ void elem_f32(unsigned char* b, int r, int c, float x) {
  *reinterpret_cast<float*>(b + off32(r, c)) = x;
}

// ---- TMA tile stores (bulk groups) ----
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, const void* src, int x, int y) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(map),
               "r"(smem_u32(src)), "r"(x), "r"(y)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

template <class OutP>
__device__ __forceinline__ void store_out(const CUtensorMap* m, const unsigned char* b, int x, int y) {
  tma_store_2d(m, b, x, y);
  if (Out<OutP>::NMAP == 2) tma_store_2d(m + 1, b + 2048, x, y);
}

// The floats x[c0 .. min(c0 + 128, n)) into this SM's L1 (one 128-byte line
// per lane of lanes 0..3; only addresses inside the n-element vector), so
// that the per-block vector reads of the epilogue do not wait on DRAM.
__device__ __forceinline__ void prefetch_l1(const float* x, int c0, int n, int lane) {
  if (x && lane < 4 && c0 + 32 * lane < n) asm volatile("prefetch.global.L1 [%0];" ::"l"(x + c0 + 32 * lane));
}

// Tile hook, run by every epilogue warp before it waits for the accumulator:
// vectors the block epilogues of tile (m0, n0) read (none by default).
template <class Epi>
__device__ __forceinline__ void tc_prefetch(const Epi&, int, int, int) {}

// Staging complete: make it visible to the async proxy, then lane 0 issues
// the stores the caller lists.
__device__ __forceinline__ void staged() {
  fence_proxy_async();
  __syncwarp();
}

// ---------------------------------------------------------------------------
// Per-functor block epilogues.  tc_skip: block outside the computed region;
// tc_in: the block needs an input block (and where it starts: x = column,
// y = row of the input matrix).
// ---------------------------------------------------------------------------

// Vt = L^T K~: acc + L[j][i] s[j] (transposed L block).
template <class OutP>
__device__ __forceinline__ bool tc_skip(const EpiVt<OutP>&, int, int) { return false; }
template <class OutP>
__device__ __forceinline__ bool tc_in(const EpiVt<OutP>& e, int i0, int j0, int& x, int& y) {
  x = i0; y = j0;
  return e.s != nullptr;
}
template <class OutP>
__device__ __forceinline__ void tc_prefetch(const EpiVt<OutP>& e, int, int n0, int lane) { prefetch_l1(e.s, n0, e.M, lane); }
template <class OutP>
__device__ __forceinline__ void tc_epi(EpiVt<OutP>& e, int i0, int j0, float (&v)[32], int lane,
                                       const unsigned char* in, unsigned char* out, const EpiMaps& maps) {
  if (e.s) {
    float lt[32];
    ld_col_f32(in, lane, lt);                     // lt[q] = L[j0 + q][i0 + lane] (zero outside M)
    const float sl = (j0 + lane < e.M) ? __ldg(e.s + j0 + lane) : 0.f;
#pragma unroll
    for (int q = 0; q < 32; ++q) v[q] = fmaf(lt[q], __shfl_sync(0xffffffffu, sl, q), v[q]);
  }
  Out<OutP>::row(out, lane, v);
  staged();
  if (lane == 0) {
    store_out<OutP>(&maps.out[0], out, j0, i0);
    bulk_commit();
  }
}

// Symmetric result on the upper region (i <= j), MODE as in EpiSym.
template <class OutP, int MODE>
__device__ __forceinline__ bool tc_skip(const EpiSym<OutP, MODE>&, int i0, int j0) { return i0 > j0 + 31; }
template <class OutP, int MODE>
__device__ __forceinline__ bool tc_in(const EpiSym<OutP, MODE>&, int, int, int&, int&) { return false; }
template <int MODE>
__device__ __forceinline__ float sym_val(float a, bool dg) {
  if (MODE == 0) return dg ? 0.5f * (a - 1.0f) : a;
  if (MODE == 1) return (dg ? 2.0f : 0.0f) - a;
  return a + (dg ? 0.5f : 0.0f);
}
template <int MODE>
__device__ __forceinline__ float sym_mirror(float a) {
  return MODE == 0 ? 0.0f : (MODE == 1 ? -a : a);
}
template <class OutP, int MODE>
__device__ __forceinline__ void tc_epi(EpiSym<OutP, MODE>& e, int i0, int j0, float (&v)[32], int lane,
                                       const unsigned char*, unsigned char* out, const EpiMaps& maps) {
  const int i = i0 + lane;
  const bool diagblk = i0 == j0;
  const bool rowin = i < e.M;
  float d[32];
  // sums over the counted triangle (weight 1 on the diagonal, 2 off it) in
  // four independent register partials, selected rather than branched
  float s0[4] = {0.f, 0.f, 0.f, 0.f}, s1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int q = 0; q < 32; ++q) {
    const int j = j0 + q;
    const bool dg = i == j;
    d[q] = sym_val<MODE>(v[q], dg);
    const bool cnt = (!diagblk || q >= lane) && rowin && j < e.M;
    const float a = v[q], w = dg ? 1.f : 2.f;
    if (MODE == 0) {
      const float t = a - (dg ? 1.f : 0.f);
      s0[q & 3] = cnt ? fmaf(w * t, t, s0[q & 3]) : s0[q & 3];
    }
    if (MODE == 1) {
      s0[q & 3] = (cnt && dg) ? s0[q & 3] + a : s0[q & 3];
      s1[q & 3] = cnt ? fmaf(w * a, a, s1[q & 3]) : s1[q & 3];
    }
  }
  if (MODE == 0) e.p0 += (s0[0] + s0[1]) + (s0[2] + s0[3]);
  if (MODE == 1) {
    e.p0 += (s0[0] + s0[1]) + (s0[2] + s0[3]);
    e.p1 += (s1[0] + s1[1]) + (s1[2] + s1[3]);
  }
  Out<OutP>::row(out, lane, d);
  if (diagblk) {
    __syncwarp();
#pragma unroll
    for (int q = 0; q < 32; ++q)
      if (q > lane) Out<OutP>::elem(out, q, lane, sym_mirror<MODE>(v[q]));
  } else {
#pragma unroll
    for (int q = 0; q < 32; ++q) Out<OutP>::elem(out + SLOT, q, lane, sym_mirror<MODE>(v[q]));
  }
  staged();
  if (lane == 0) {
    store_out<OutP>(&maps.out[0], out, j0, i0);
    if (!diagblk) store_out<OutP>(&maps.out[0], out + SLOT, i0, j0);
    bulk_commit();
  }
}

// NG update of L: L_ij <- L_ij - gamma acc on the lower region; the padded
// FP32 copy by TMA, the caller's L (leading dimension M) by coalesced stores
// read back from the staging block.
__device__ __forceinline__ bool tc_skip(const EpiLupd&, int i0, int j0) { return j0 > i0 + 31; }
__device__ __forceinline__ bool tc_in(const EpiLupd&, int i0, int j0, int& x, int& y) {
  x = j0; y = i0;
  return true;
}
__device__ __forceinline__ void tc_epi(EpiLupd& e, int i0, int j0, float (&v)[32], int lane, const unsigned char* in,
                                       unsigned char* out, const EpiMaps& maps) {
  const float g = *e.gamma;
  const int i = i0 + lane;
  float old[32];
  ld_row_f32(in, lane, old);
#pragma unroll
  for (int q = 0; q < 32; ++q) v[q] = (j0 + q <= i) ? old[q] - g * v[q] : 0.f;
  row_f32(out, lane, v);
  staged();
  if (lane == 0) {
    tma_store_2d(&maps.out[0], out, j0, i0);
    bulk_commit();
  }
  // all 32 shared-memory reads before the first global store (the compiler
  // cannot reorder them across stores that might alias)
  const int j = j0 + lane, M = e.M;
  float* Lout = e.Lout;
  float col[32];
#pragma unroll
  for (int r = 0; r < 32; ++r) col[r] = *reinterpret_cast<const float*>(out + off32(r, lane));
#pragma unroll
  for (int r = 0; r < 32; ++r) {
    const int ii = i0 + r;
    if (j <= ii && ii < M && j < M) Lout[(size_t)ii * M + j] = col[r];
  }
}

// Plain store of a full result.
template <class OutP>
__device__ __forceinline__ bool tc_skip(const EpiStore<OutP>&, int, int) { return false; }
template <class OutP>
__device__ __forceinline__ bool tc_in(const EpiStore<OutP>&, int, int, int&, int&) { return false; }
template <class OutP>
__device__ __forceinline__ void tc_epi(EpiStore<OutP>&, int i0, int j0, float (&v)[32], int lane,
                                       const unsigned char*, unsigned char* out, const EpiMaps& maps) {
  Out<OutP>::row(out, lane, v);
  staged();
  if (lane == 0) {
    store_out<OutP>(&maps.out[0], out, j0, i0);
    bulk_commit();
  }
}

// Transposed store: the block goes out as its transpose (column stores into
// the staging slot, as the mirrored blocks of the symmetric results).
template <class OutP>
__device__ __forceinline__ bool tc_skip(const EpiStoreT<OutP>&, int, int) { return false; }
template <class OutP>
__device__ __forceinline__ bool tc_in(const EpiStoreT<OutP>&, int, int, int&, int&) { return false; }
template <class OutP>
__device__ __forceinline__ void tc_epi(EpiStoreT<OutP>&, int i0, int j0, float (&v)[32], int lane,
                                       const unsigned char*, unsigned char* out, const EpiMaps& maps) {
#pragma unroll
  for (int q = 0; q < 32; ++q) Out<OutP>::elem(out, q, lane, v[q]);
  staged();
  if (lane == 0) {
    store_out<OutP>(&maps.out[0], out, i0, j0);
    bulk_commit();
  }
}

// P on the lower region, mirrored: FP32 (maps.out[0]) and operand-precision
// copies (maps.out[1..]); sum_i s_i P_ii and <P, Psi>.
template <class OutP>
__device__ __forceinline__ bool tc_skip(const EpiP<OutP>&, int i0, int j0) { return j0 > i0 + 31; }
template <class OutP>
__device__ __forceinline__ bool tc_in(const EpiP<OutP>& e, int i0, int j0, int& x, int& y) {
  x = j0; y = i0;
  return e.Psi != nullptr;
}
template <class OutP>
__device__ __forceinline__ void tc_prefetch(const EpiP<OutP>& e, int m0, int n0, int lane) {
  if (m0 == n0) prefetch_l1(e.s, m0, e.M, lane);
}
template <class OutP>
__device__ __forceinline__ void tc_epi(EpiP<OutP>& e, int i0, int j0, float (&v)[32], int lane,
                                       const unsigned char* in, unsigned char* out, const EpiMaps& maps) {
  const int i = i0 + lane;
  const bool diagblk = i0 == j0;
  if (i < e.M) {
    if (diagblk) {                                   // P_ii sits at q == lane
      float pii = 0.f;
#pragma unroll
      for (int q = 0; q < 32; ++q) pii = q == lane ? v[q] : pii;
      e.p0 = fmaf(__ldg(e.s + i), pii, e.p0);
    }
    if (e.Psi) {
      float ps[32];
      ld_row_f32(in, lane, ps);
      float s1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const int j = j0 + q;
        const bool cnt = j <= i && j < e.M;
        s1[q & 3] = cnt ? fmaf((j == i ? 1.f : 2.f) * v[q], ps[q], s1[q & 3]) : s1[q & 3];
      }
      e.p1 += (s1[0] + s1[1]) + (s1[2] + s1[3]);
    }
  }
  row_f32(out, lane, v);
  Out<OutP>::row(out + SLOT, lane, v);
  if (diagblk) {
    __syncwarp();
#pragma unroll
    for (int q = 0; q < 32; ++q)
      if (q < lane) {
        elem_f32(out, q, lane, v[q]);
        Out<OutP>::elem(out + SLOT, q, lane, v[q]);
      }
  } else {
#pragma unroll
    for (int q = 0; q < 32; ++q) {
      elem_f32(out + 2 * SLOT, q, lane, v[q]);
      Out<OutP>::elem(out + 3 * SLOT, q, lane, v[q]);
    }
  }
  staged();
  if (lane == 0) {
    tma_store_2d(&maps.out[0], out, j0, i0);
    store_out<OutP>(&maps.out[1], out + SLOT, j0, i0);
    if (!diagblk) {
      tma_store_2d(&maps.out[0], out + 2 * SLOT, i0, j0);
      store_out<OutP>(&maps.out[1], out + 3 * SLOT, i0, j0);
    }
    bulk_commit();
  }
}

// G_Kuu = G_K~ + P/2 - v v^T / 2 on the lower region, mirrored; ds.
__device__ __forceinline__ bool tc_skip(const EpiGK&, int i0, int j0) { return j0 > i0 + 31; }
__device__ __forceinline__ bool tc_in(const EpiGK&, int i0, int j0, int& x, int& y) {
  x = j0; y = i0;
  return true;
}
__device__ __forceinline__ void tc_prefetch(const EpiGK& e, int m0, int n0, int lane) {
  prefetch_l1(e.v, m0, e.M, lane);
  prefetch_l1(e.v, n0, e.M, lane);
  if (m0 == n0) prefetch_l1(e.s, m0, e.M, lane);
}
__device__ __forceinline__ void tc_epi(EpiGK& e, int i0, int j0, float (&v)[32], int lane, const unsigned char* in,
                                       unsigned char* out, const EpiMaps& maps) {
  const int i = i0 + lane;
  const bool diagblk = i0 == j0;
  float p[32];
  ld_row_f32(in, lane, p);
  const float vi = i < e.M ? __ldg(e.v + i) : 0.f;
  const float vc = (j0 + lane) < e.M ? __ldg(e.v + j0 + lane) : 0.f;
  float g[32];
#pragma unroll
  for (int q = 0; q < 32; ++q) {
    const float vj = __shfl_sync(0xffffffffu, vc, q);
    g[q] = -v[q] + 0.5f * p[q] - 0.5f * vi * vj;
  }
  if (diagblk) {                                     // G_ii term at q == lane
    float vii = 0.f;
#pragma unroll
    for (int q = 0; q < 32; ++q) vii = q == lane ? v[q] : vii;
    if (i < e.M) e.ds[i] = -vii + 0.5f / e.s[i];
  }
  row_f32(out, lane, g);
  if (diagblk) {
    __syncwarp();
#pragma unroll
    for (int q = 0; q < 32; ++q)
      if (q < lane) elem_f32(out, q, lane, g[q]);
  } else {
#pragma unroll
    for (int q = 0; q < 32; ++q) elem_f32(out + SLOT, q, lane, g[q]);
  }
  staged();
  if (lane == 0) {
    tma_store_2d(&maps.out[0], out, j0, i0);
    if (!diagblk) tma_store_2d(&maps.out[0], out + SLOT, i0, j0);
    bulk_commit();
  }
}

}  // namespace etc
