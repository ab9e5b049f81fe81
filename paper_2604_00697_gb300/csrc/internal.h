// Host-side declarations shared by the translation units of the library.
#pragma once
#include "common.cuh"

// Tile tables and stream for the M x M GEMMs of one handle.  All matrices are
// Mp x Mp row-major with ld = Mp (Mp = M rounded up to 128, zero padded).
struct GemmCtx {
  int Mp;
  cudaStream_t st;
  int* err;       // device error word of the handle
  // Tables (device memory).  Regions and K ranges (L lower, Lt = L^T upper):
  //  vt     : full,  K [m0, Mp)          Lt S       (S symmetric)
  //  sym_in : upper, K [n0, Mp)          V Lt^T     = L^T S L
  //  lupd   : lower, K [n0, m0 + BM)     L Phi      (Phi lower)
  //  ls     : full,  K [0, m0 + BM)      L S
  //  out    : lower, K [0, n0 + BN)      Y L^T      = L S L^T
  //  psi    : upper, K given at launch   Kuf Kuf^T
  Tile *tt_vt, *tt_sym_in, *tt_lupd, *tt_ls, *tt_out, *tt_psi;
  int nt_vt, nt_sym_in, nt_lupd, nt_ls, nt_out, nt_psi;
};

// Process-wide count of kernel launches issued by the library (svgp_api.cu).
void svgp_note_launch();

// FP32 SIMT launchers (gemm_simt.cu).
void simt_vt(const GemmCtx& g, const float* Lt, const float* Kuu, EpiVt<float> e);
void simt_sym_ng(const GemmCtx& g, const float* Vt, const float* Lt, EpiSym<float, 0> e);
void simt_sym_fwd(const GemmCtx& g, const float* Vt, const float* Lt, EpiSym<float, 1> e);
void simt_sym_bwd(const GemmCtx& g, const float* Vt, const float* Lt, EpiSym<float, 2> e);
void simt_lupd(const GemmCtx& g, const float* L, const float* PhiT, EpiLupd e);
void simt_ls(const GemmCtx& g, const float* L, const float* S, EpiStore<float> e);
void simt_p(const GemmCtx& g, const float* Y, const float* L, EpiP<float> e);
void simt_gk(const GemmCtx& g, const float* Y, const float* L, EpiGK e);
void simt_psi(const GemmCtx& g, const KufGen& kg, int B, EpiPsi e);
void simt_w(const GemmCtx& g, const float* P, const WEpi& we);
void simt_init_attributes();

// tcgen05 BF16 launchers (gemm_tc.cu).  Return false when the tensor-core
// path is not available for this device.
bool tc_available();
void tc_init_attributes();
bool tc_vt(const GemmCtx& g, const bf16* Lt, const bf16* Kuu, EpiVt<bf16> e);
bool tc_sym_ng(const GemmCtx& g, const bf16* Vt, const bf16* Lt, EpiSym<bf16, 0> e);
bool tc_sym_fwd(const GemmCtx& g, const bf16* Vt, const bf16* Lt, EpiSym<bf16, 1> e);
bool tc_sym_bwd(const GemmCtx& g, const bf16* Vt, const bf16* Lt, EpiSym<bf16, 2> e);
bool tc_lupd(const GemmCtx& g, const bf16* L, const bf16* PhiT, EpiLupd e);
bool tc_ls(const GemmCtx& g, const bf16* L, const bf16* S, EpiStore<bf16> e);
bool tc_p(const GemmCtx& g, const bf16* Y, const bf16* L, EpiP<bf16> e);
bool tc_gk(const GemmCtx& g, const bf16* Y, const bf16* L, EpiGK e);
bool tc_psi(const GemmCtx& g, const KufGen& kg, int B, EpiPsi e);
bool tc_w(const GemmCtx& g, const bf16* P, const WEpi& we);

// Miscellaneous kernels (kernels_misc.cu).
void k_prep_coords(const float* Z, const float* X, const float* ell, int M, int Mp, int B, int D,
                   float* Zs, float* Xs, cudaStream_t st);
template <class LoT>
void k_kuu(const float* Zs, int M, int Mp, int D, const float* sf2, float* Kf, LoT* Klo,
           cudaStream_t st);
template <class LoT>
void k_prep_L(const float* Lin, int M, int Mp, float* Lf, LoT* Llo, LoT* Ltlo, double* red,
              cudaStream_t st);
void k_gemv(const float* A, int Mp, int M, const float* x, float alpha, const float* x2, float beta,
            float* y, const float* dotw, double* dot_out, cudaStream_t st);
void k_mu(const float* Zs, const float* Xs, int M, int B, int D, const float* sf2, const float* v,
          float* mu, cudaStream_t st);
void k_pointwise_gauss(const float* y, const float* mu, const float* noise, int B, float* g,
                       double* red, cudaStream_t st);
void k_kg(const float* Zs, const float* Xs, int M, int Mp, int B, int D, const float* sf2,
          const float* g, float* Kg, cudaStream_t st);
template <class LoT>
void k_gp_assemble(const float* Kuu, const float* Psi, const float* Kg, const float* m,
                   const float* w, const float* noise, float c, int M, int Mp, LoT* out,
                   cudaStream_t st);
void k_kuu_bwd(const float* GKuu, const float* Kuu, const float* Zs, int M, int Mp, int D,
               float* rowacc_u, double* red, cudaStream_t st);
void k_logs(const float* s, int M, double* red, cudaStream_t st);
void k_grad_finalize(const float* rowacc_f, const float* rowacc_u, const float* ell, int M, int D,
                     float* dZ, double* acc_ell, double* red, cudaStream_t st);
void k_terms_finalize(const double* red, const double* acc_ell, const float* sf2, const float* noise,
                      const float* ell, int M, int D, int B, double N, double* terms,
                      float* dsf2, float* dnoise, float* dell, int* errword, cudaStream_t st);
void k_predict_finalize(const float* colsum, const float* sf2, const float* noise, int Ns,
                        int include_noise, float* var, cudaStream_t st);
void k_adam(float* raw, float* cons, const float* grad, float* m1, float* m2, int* step,
            const float* hyper, const float* zbeta1, int M, int D, cudaStream_t st);
void k_ng_check(const double* red, int M, double eps, int* done, int* iters, double* resid,
                cudaStream_t st);
