// Host-side declarations shared by the translation units of the library.
#pragma once
#include "common.cuh"

// Tile tables of the M x M contractions.  All matrices are Mp x Mp row-major
// with ld = Mp (Mp = M rounded up to 128, zero padded).  L is lower
// triangular, Lt = L^T upper triangular; regions and K ranges:
enum TileTable {
  TT_VT = 0,      // full,  K [m0, Mp)        Lt S        (S symmetric)
  TT_SYM_IN = 1,  // upper, K [n0, Mp)        V Lt^T      = L^T S L
  TT_LUPD = 2,    // lower, K [n0, m0 + BM)   L Phi       (Phi lower)
  TT_LS = 3,      // full,  K [0, m0 + BM)    L S
  TT_OUT = 4,     // lower, K [0, n0 + BN)    Y L^T       = L S L^T
  TT_PSI = 5,     // upper, K given at launch Kuf Kuf^T
  TT_COUNT = 6
};

struct GemmCtx {
  int Mp;
  cudaStream_t st;
  int* err;        // device error word of the handle
  bool split;      // tensor-core operands are hi/lo BF16 pairs (lo at +Mp*Mp)
  Tile* tt[TT_COUNT];
  int nt[TT_COUNT];
  // tensor-core schedule: CTA c of a launch of ncta[t] CTAs processes the
  // tiles tt[t][toff[t][c] .. toff[t][c + 1])
  int* toff[TT_COUNT];
  int ncta[TT_COUNT];
};

// Process-wide count of kernel launches issued by the library (svgp_api.cu).
void svgp_note_launch();

// FP32 SIMT contractions (gemm_simt.cu): acc = A B^T over table `tab`.
template <class Epi>
void simt_gemm(const GemmCtx& g, int tab, const float* A, const float* B, const Epi& e);
void simt_psi(const GemmCtx& g, const KufGen& kg, int B, EpiPsi e);
void simt_w(const GemmCtx& g, const float* P, const WEpi& we);
void simt_init_attributes();

// tcgen05 BF16 contractions (gemm_tc.cu): acc = A B^T over table `tab`; A and
// B point at the hi part (lo at +Mp*Mp when g.split).  Return false when the
// tensor-core path is unavailable.
bool tc_available();
int tc_num_sms();
void tc_init_attributes();
template <class Epi>
bool tc_gemm(const GemmCtx& g, int tab, const bf16* A, const bf16* B, const Epi& e);

// Tensor-core Kuf-producer contractions (gemm_kuf_tc.cu): split coordinates
// of the generator (64 BF16 per point: row role [hi, hi, lo], k role
// [hi, lo, hi]) and per-point offsets c = -1/2 log2(e) |p|^2.
struct KufTC {
  bf16 *ZR, *ZK, *XR, *XK;
};
bool tc_kuf_supported(int D);
void tc_kuf_init_attributes();
void k_kuf_prep(const float* Zs, const float* Xs, int M, int Mp, int B, int Bp, int D, const float* sf2,
                const KufTC& t, cudaStream_t st);
bool tc_psi(const GemmCtx& g, const KufGen& kg, const KufTC& t, int B, EpiPsi e);
// W = P Kuf with its fused epilogue.  Gradient mode (we.rowacc != null):
// writes per-CTA partial rows rowpart[p][k][i] (p < returned count, k < 2D+1,
// i < Mp) instead of rowacc; variance mode returns 0.  -1: not supported.
int tc_w(const GemmCtx& g, const bf16* P, const KufTC& t, const WEpi& we, float* rowpart);
int tc_w_groups(int Mp, int B);
void tc_w_init_attributes();
// out[r] = sum_k Kuf(r, k) w_k for r < nrows, k < nk, from the row-role vectors
// of the row points and the k-role vectors of the k points (kuf_prep).
bool tc_kuf_gemv(const bf16* Rrole, int nrows, const bf16* Krole, int nk, const float* w, float* out, int* errword,
                 cudaStream_t st);
void tc_gemv_init_attributes();

// Miscellaneous kernels (kernels_misc.cu).  OutP is float*, bf16* or SplitPtr.
void k_prep_coords(const float* Z, const float* X, const float* ell, int M, int Mp, int B, int D,
                   float* Zs, float* Xs, cudaStream_t st);
template <class OutP>
void k_kuu(const float* Zs, int M, int Mp, int D, const float* sf2, float* Kf, OutP Klo, bool has_lo,
           cudaStream_t st);
template <class OutP>
void k_prep_L(const float* Lin, int M, int Mp, float* Lf, OutP Llo, OutP Ltlo, double* logdet,
              cudaStream_t st);
void k_gemv(const float* A, int Mp, int M, const float* x, float alpha, const float* x2, float beta,
            float* y, const float* dotw, double* dot_out, cudaStream_t st);
void k_mu(const float* Zs, const float* Xs, int M, int B, int D, const float* sf2, const float* v,
          float* mu, cudaStream_t st);
void k_pointwise_gauss(const float* y, const float* mu, const float* noise, int B, float* g,
                       double* red, cudaStream_t st);
void k_kg(const float* Zs, const float* Xs, int M, int Mp, int B, int D, const float* sf2,
          const float* g, float* Kg, cudaStream_t st);
template <class OutP>
void k_gp_assemble(const float* Kuu, const float* Psi, const float* Kg, const float* m,
                   const float* w, const float* noise, float c, int M, int Mp, OutP out,
                   cudaStream_t st);
void k_kuu_bwd(const float* GKuu, const float* Kuu, const float* Zs, int M, int Mp, int D,
               float* rowacc_u, double* red, cudaStream_t st);
void k_logs(const float* s, int M, double* red, cudaStream_t st);
void k_grad_finalize(const float* rowacc_f, const float* rowacc_u, const float* rowpart, int nparts, int Mp,
                     const float* ell, int M, int D, float* dZ, double* acc_ell, double* red, cudaStream_t st);
void k_terms_finalize(const double* red, const double* acc_ell, const float* sf2, const float* noise,
                      const float* ell, int M, int D, int B, double N, double* terms,
                      float* dsf2, float* dnoise, float* dell, int* errword, cudaStream_t st);
void k_predict_finalize(const float* colsum, const float* sf2, const float* noise, int Ns,
                        int include_noise, float* var, cudaStream_t st);
void k_adam(float* raw, float* cons, const float* grad, float* m1, float* m2, int* step,
            const float* hyper, const float* zbeta1, int M, int D, cudaStream_t st);
void k_ng_check(const double* red, int M, double eps, int* done, int* iters, double* resid,
                cudaStream_t st);
