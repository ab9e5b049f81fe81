// Prediction that allocates no device memory: the same FP32 kernels as
// svgp_predict on a handle created with SVGP_FP32, with all of their scratch
// carved out of one file-scope device array instead of a handle's workspace.
#include <string.h>

#include "common.cuh"
#include "internal.h"

namespace {

constexpr int NA_MAXM = 256;      // inducing points (padded size Mp <= 256)
constexpr int NA_MAXN = 4096;     // test inputs per call
constexpr int NA_MAXD = SVGP_MAXD;
constexpr int NA_TAB = 4;         // tiles per table at Mp <= 256 with 128 x 128 tiles

// Offsets (bytes, 256-aligned) of the pieces of the scratch array.
constexpr size_t al(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t MAT = sizeof(float) * NA_MAXM * NA_MAXM;
constexpr size_t OFF_ZS = 0;
constexpr size_t OFF_XS = al(OFF_ZS + sizeof(float) * NA_MAXM * NA_MAXD);
constexpr size_t OFF_KUU = al(OFF_XS + sizeof(float) * NA_MAXN * NA_MAXD);
constexpr size_t OFF_LF = OFF_KUU + MAT;
constexpr size_t OFF_LLO = OFF_LF + MAT;
constexpr size_t OFF_LT = OFF_LLO + MAT;
constexpr size_t OFF_V = OFF_LT + MAT;
constexpr size_t OFF_S = OFF_V + MAT;
constexpr size_t OFF_Y = OFF_S + MAT;
constexpr size_t OFF_P = OFF_Y + MAT;
constexpr size_t OFF_VEC = OFF_P + MAT;                          // v (MAXM floats)
constexpr size_t OFF_COL = al(OFF_VEC + sizeof(float) * NA_MAXM);
constexpr size_t OFF_RED = al(OFF_COL + sizeof(float) * NA_MAXN);
constexpr size_t OFF_ERR = al(OFF_RED + sizeof(double) * RED_COUNT);
constexpr size_t OFF_TAB = al(OFF_ERR + sizeof(int));        // tables for Mp = 128, then Mp = 256
constexpr size_t TAB_SET = sizeof(Tile) * TT_COUNT * NA_TAB;
constexpr size_t NA_BYTES = al(OFF_TAB + 2 * TAB_SET);

// The scratch itself (about 2.7 MB; every GPU that loads the library holds
// it until the process exits).
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

// Tile tables for Mp = 128 * nb (nb = 1 or 2), in the layout of
// make_tiles(): VT full / K [m0, Mp); SYM_IN upper / K [n0, Mp);
// LS full / K [0, m0 + 128); OUT lower / K [0, n0 + 128).  Built on the host.
void na_tables(Tile* tab, int nb) {
  const int Mp = 128 * nb;
  int c[TT_COUNT] = {0};
  for (int a = 0; a < nb; ++a)
    for (int b = 0; b < nb; ++b) {
      const int m0 = 128 * a, n0 = 128 * b;
      tab[TT_VT * NA_TAB + c[TT_VT]++] = Tile{m0, n0, m0, Mp};
      if (m0 <= n0) tab[TT_SYM_IN * NA_TAB + c[TT_SYM_IN]++] = Tile{m0, n0, n0, Mp};
      tab[TT_LS * NA_TAB + c[TT_LS]++] = Tile{m0, n0, 0, m0 + 128};
      if (m0 >= n0) tab[TT_OUT * NA_TAB + c[TT_OUT]++] = Tile{m0, n0, 0, n0 + 128};
    }
}

struct NaDevice {
  unsigned char* base;   // device address of g_noalloc_scratch on this device
};
NaDevice g_na[64];

}  // namespace

extern "C" svgp_status svgp_predict_noalloc(const svgp_params* p, int M, int D, const float* Xs, int Ns,
                                            float* mean, float* var, int include_noise, void* cuda_stream) {
  if (!p || !p->Z || !p->ell || !p->sf2 || !p->noise || !p->m || !p->s || !p->L || !Xs || !mean || !var)
    return SVGP_ERR_INVALID_ARG;
  if (M < 1 || M > NA_MAXM || D < 1 || D > NA_MAXD || Ns < 1 || Ns > NA_MAXN) return SVGP_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SVGP_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  NaDevice& nd = g_na[dev];
  if (!nd.base) {
    // One-time set-up on this device (must not run inside a stream capture):
    // the host-side symbol is only a stand-in, the kernels need its device
    // address; the tile tables of both padded sizes are copied in once, so no
    // call depends on the work an earlier call enqueued; the FP32 kernels need
    // their shared-memory limits raised.
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return SVGP_ERR_CUDA;
    Tile tabs[2 * TT_COUNT * NA_TAB];
    memset(tabs, 0, sizeof(tabs));
    na_tables(tabs, 1);
    na_tables(tabs + TT_COUNT * NA_TAB, 2);
    if (cudaMemcpyToSymbol(g_noalloc_scratch, tabs, sizeof(tabs), OFF_TAB, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess)
      return SVGP_ERR_CUDA;
    simt_init_attributes();
    nd.base = reinterpret_cast<unsigned char*>(ptr);
  }
  unsigned char* b = nd.base;
  const int Mp = (M + 127) / 128 * 128;
  const int nb = Mp / 128;
  Tile* tab = reinterpret_cast<Tile*>(b + OFF_TAB + (nb - 1) * TAB_SET);
  GemmCtx g;
  memset(&g, 0, sizeof(g));
  g.Mp = Mp;
  g.st = st;
  g.err = reinterpret_cast<int*>(b + OFF_ERR);
  g.split = false;
  for (int t = 0; t < TT_COUNT; ++t) g.tt[t] = tab + t * NA_TAB;
  g.nt[TT_VT] = nb * nb;
  g.nt[TT_SYM_IN] = nb * (nb + 1) / 2;
  g.nt[TT_LS] = nb * nb;
  g.nt[TT_OUT] = nb * (nb + 1) / 2;
  float* Zs = reinterpret_cast<float*>(b + OFF_ZS);
  float* Xsc = reinterpret_cast<float*>(b + OFF_XS);
  float* Kuu = reinterpret_cast<float*>(b + OFF_KUU);
  float* Lf = reinterpret_cast<float*>(b + OFF_LF);
  float* Llo = reinterpret_cast<float*>(b + OFF_LLO);
  float* Lt = reinterpret_cast<float*>(b + OFF_LT);
  float* V = reinterpret_cast<float*>(b + OFF_V);
  float* S = reinterpret_cast<float*>(b + OFF_S);
  float* Y = reinterpret_cast<float*>(b + OFF_Y);
  float* P = reinterpret_cast<float*>(b + OFF_P);
  float* v = reinterpret_cast<float*>(b + OFF_VEC);
  float* colsum = reinterpret_cast<float*>(b + OFF_COL);
  double* red = reinterpret_cast<double*>(b + OFF_RED);
  // The array keeps the previous call's contents: clear the accumulators.
  cudaMemsetAsync(red, 0, sizeof(double) * RED_COUNT, st);
  cudaMemsetAsync(colsum, 0, sizeof(float) * Ns, st);
  // Same sequence as svgp_predict on an FP32 handle.
  k_prep_coords(p->Z, Xs, p->ell, M, Mp, Ns, D, Zs, Xsc, st);
  k_kuu(Zs, M, Mp, D, p->sf2, Kuu, (float*)nullptr, false, st);
  k_prep_L(p->L, M, Mp, Lf, Llo, Lt, red + RED_LOGDETL, st);
  simt_gemm(g, TT_VT, Lt, Kuu, EpiVt<float*>{V, Mp, Lf, p->s, M, nullptr});
  simt_gemm(g, TT_SYM_IN, V, Lt, EpiSym<float*, 1>{S, Mp, M, red, nullptr});
  simt_gemm(g, TT_LS, Llo, S, EpiStore<float*>{Y, Mp, nullptr});
  simt_gemm(g, TT_OUT, Y, Llo, EpiP<float*>{P, P, Mp, M, p->s, nullptr, red});
  k_gemv(P, Mp, M, p->m, 1.f, nullptr, 0.f, v, nullptr, nullptr, st);
  k_mu(Zs, Xsc, M, Ns, D, p->sf2, v, mean, st);
  WEpi we{KufGen{Zs, Xsc, D, M, Ns, p->sf2}, nullptr, nullptr, nullptr, nullptr, 0.f, nullptr, colsum};
  simt_w(g, P, we);
  k_predict_finalize(colsum, p->sf2, p->noise, Ns, include_noise, var, st);
  return cudaGetLastError() == cudaSuccess ? SVGP_OK : SVGP_ERR_CUDA;
}
