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
  TT_FULL = 6,    // full,  K [0, Mp)         general products (Prop. 3 gap)
  // tall-skinny products A X of the P-free bound, output columns [0, Np) only
  // (Np set per call), X stored transposed (one row per column of X)
  TT_RL = 7,      // K [0, m0 + BM)           A = L
  TT_RLT = 8,     // K [m0, Mp)               A = L^T
  TT_RF = 9,      // K [0, Mp)                A = Kuu or K~
  TT_COUNT = 10
};

// One work item of the persistent tensor-core GEMM: an output tile and its K
// range, whole (role TC_WHOLE) or one of two K chunks of a split tile.  The
// producer chunk (TC_PRODUCER) writes its FP32 partial sums to workspace slot
// `slot` and counts itself done; the owner chunk (TC_OWNER) waits for that
// count, adds the partial and runs the epilogue.
enum { TC_WHOLE = 0, TC_PRODUCER = 1, TC_OWNER = 2 };
struct TcTile {
  int m0, n0, k0, k1, role, slot;
};

struct GemmCtx {
  int Mp;
  cudaStream_t st;
  int* err;        // device error word of the handle
  bool split;      // tensor-core operands are hi/lo BF16 pairs (lo at +Mp*Mp)
  Tile* tt[TT_COUNT];
  int nt[TT_COUNT];
  // tensor-core schedule: CTA c of a launch of ncta[t] CTAs processes the
  // items tct[t][toff[t][c] .. toff[t][c + 1])
  TcTile* tct[TT_COUNT];
  int* toff[TT_COUNT];
  int ncta[TT_COUNT];
  // split-K workspace: 128 x 128 FP32 partial per slot, and per slot the
  // producer's done count and the owner warps' read count (zero between launches)
  float* kpart;
  int* kflag;
  int nslot;
};

// Process-wide count of kernel launches issued by the library (svgp_api.cu).
void svgp_note_launch();

// FP32 SIMT contractions (gemm_simt.cu): acc = A B^T over table `tab`.
template <class Epi>
void simt_gemm(const GemmCtx& g, int tab, const float* A, const float* B, const Epi& e);
// hw (may be null): per-point weights h_n; the result is then
// Kuf diag(|h|) Kuf^T (both generated operands scaled by sqrt|h_n|).
void simt_psi(const GemmCtx& g, const KufGen& kg, int B, EpiPsi e, const float* hw);
void simt_w(const GemmCtx& g, const float* P, const WEpi& we);
void simt_init_attributes();

// tcgen05 BF16 contractions (gemm_tc.cu): acc = A B^T over table `tab`; A and
// B point at the hi part (lo at +Mp*Mp when g.split).  Return false when the
// tensor-core path is unavailable.
bool tc_available();
// One-block probe whose bounded mbarrier wait runs out (raises ERRBIT_TIMEOUT).
void tc_wait_probe(int* errword, cudaStream_t st);
int tc_num_sms();
void tc_init_attributes();
template <class Epi>
bool tc_gemm(const GemmCtx& g, int tab, const bf16* A, const bf16* B, const Epi& e, const bf16* B3 = nullptr);

// Tensor-core Kuf-producer contractions (gemm_kuf_tc.cu): split coordinates
// of the generator (64 BF16 per point: row role [hi, hi, lo], k role
// [hi, lo, hi]) and per-point offsets c = -1/2 log2(e) |p|^2.
struct KufTC {
  bf16 *ZR, *ZK, *XR, *XK;
  bf16* XKh;   // k role of x with the constant raised by 1/2 log2|h_n| (probit Psi weights)
};
bool tc_kuf_supported(int D);
void tc_kuf_init_attributes();
void k_kuf_prep(const float* Zs, const float* Xs, int M, int Mp, int B, int Bp, int D, const float* sf2,
                const KufTC& t, cudaStream_t st);
// K-role vectors of the x points with the per-point weight sqrt|h_n| folded
// into the constant (|h_n| < 1e-30 gives the value 0), for the weighted Psi.
void k_kuf_prep_weighted(const float* Xs, int B, int Bp, int D, const float* sf2, const float* h, bf16* XKh,
                         cudaStream_t st);
// Psi = Kxf Kxf^T with the k-role vectors Kk of the x points (t.XK: Kuf Kuf^T;
// t.XKh: Kuf diag(|h|) Kuf^T).
bool tc_psi(const GemmCtx& g, const KufGen& kg, const KufTC& t, const bf16* Kk, int B, EpiPsi e);
// W = P Kuf with its fused epilogue.  Gradient mode (we.rowacc != null):
// writes per-CTA partial rows rowpart[p][k][i] (p < returned count, k < 2D+1,
// i < Mp) instead of rowacc; variance mode returns 0.  -1: not supported.
int tc_w(const GemmCtx& g, const bf16* P, const KufTC& t, const WEpi& we, float* rowpart);
int tc_w_groups(int Mp, int B, bool split, int D);
void tc_w_init_attributes();
// out[r] = sum_k Kuf(r, k) w_k for r < nrows, k < nk, from the row-role vectors
// of the row points and the k-role vectors of the k points (kuf_prep); the
// kernel accumulates, so out is zeroed first unless out_zeroed.
bool tc_kuf_gemv(const bf16* Rrole, int nrows, const bf16* Krole, int nk, const float* w, float* out, bool out_zeroed, int* errword,
                 cudaStream_t st);
void tc_gemv_init_attributes();

// Miscellaneous kernels (kernels_misc.cu).  OutP is float*, bf16* or SplitPtr.
// With logs != null also *logs += sum_i log s[i] (i < M).
void k_prep_coords(const float* Z, const float* X, const float* ell, int M, int Mp, int B, int D,
                   float* Zs, float* Xs, cudaStream_t st, const float* s = nullptr, double* logs = nullptr);
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
// K~ = Kuu + diag(s) in FP32 (Mp x Mp, zero padding).
void k_kt_f32(const float* Kuu, const float* s, int M, int Mp, float* Kt, cudaStream_t st);
// Prop. 3 gap from red[RED_GAPDOT] = <N N^T, Psi>: G = dot / sigma2 with
// sigma2 = sigma2_host, or min_i s_i when sigma2_host <= 0.  Writes *gap (may
// be null); with eps > 0 sets *done when G <= 2 noise eps.
void k_gap_check(const double* red, const float* s, int M, double sigma2_host, const float* noise, double eps,
                 int* done, double* gap, cudaStream_t st);
// Zero up to ZERO_MAX device ranges (byte counts, multiples of 4; null
// pointers skipped) in one launch (a kernel rather than memset nodes keeps
// the step's launches programmatic).
constexpr int ZERO_MAX = 8;
struct ZeroRange { void* p; size_t bytes; };
void k_zero_n(cudaStream_t st, const ZeroRange* r, int n);
void k_zero(cudaStream_t st, void* p0, size_t b0, void* p1 = nullptr, size_t b1 = 0, void* p2 = nullptr,
            size_t b2 = 0);
// y = alpha (x + beta x2), n elements.
void k_axpy(const float* x, float alpha, const float* x2, float beta, float* y, int n, cudaStream_t st);
void k_pointwise_gauss(const float* y, const float* mu, const float* noise, int B, float* g,
                       double* red, cudaStream_t st);

// Bernoulli-probit likelihood (probit.cu).  Gauss-Hermite rule for exp(-t^2).
constexpr int GH_MAX = 32;
struct GHRule {
  int n;
  double t[GH_MAX], w[GH_MAX];   // nodes, weights / sqrt(pi)
};
// Host: n nodes and weights of the rule (ascending); false if n is out of [1, 64].
bool gauss_hermite_rule(int n, double* t, double* w);
// Per point: sigma_n^2 = max(sf2 - colsum_n, 0), E_n, g_n, h_n; sums of E_n,
// h_n, sigma_n^2 and the clamp count into red.
void k_pointwise_probit(const float* y, const float* mu, const float* colsum, const float* sf2, int B,
                        const GHRule& gh, float* g, float* h, double* red, cudaStream_t st);
void k_kg(const float* Zs, const float* Xs, int M, int Mp, int B, int D, const float* sf2,
          const float* g, float* Kg, cudaStream_t st);
// noise == null (probit): Psi holds Kuf diag(|h|) Kuf^T and enters with
// coefficient c; otherwise Psi = Kuf Kuf^T with c / (2 noise).  m == null:
// the bound without the preconditioner (no m~ terms in G_P).
template <class OutP>
void k_gp_assemble(const float* Kuu, const float* Psi, const float* Kg, const float* m,
                   const float* w, const float* noise, float c, int M, int Mp, OutP out,
                   cudaStream_t st);
void k_kuu_bwd(const float* GKuu, const float* Kuu, const float* Zs, int M, int Mp, int D,
               float* rowacc_u, double* red, cudaStream_t st);
void k_logs(const float* s, int M, double* red, cudaStream_t st);
void k_grad_finalize(const float* rowacc_f, const float* rowacc_u, const float* rowpart, int nparts, int Mp,
                     const float* ell, int M, int D, float* dZ, double* acc_ell, double* red, cudaStream_t st);
// Hutchinson sums of the KL traces into red[RED_HKT], red[RED_HW1],
// red[RED_HX4] for K probes Z (M x K); buffers of M x K floats (hutchinson.cu).
void k_hutchinson(const float* Lf, const float* Kuu, const float* s, int M, int Mp, const float* Z, int K,
                  float* bufA, float* bufB, float* bufC, double* red, cudaStream_t st);
// The bound's data-term inputs without P (hutchinson.cu): v = P m~ (m~ when
// precond is false) and, per point, k_n^T P k_n into colq[n] and summed into
// red[RED_PPSI], from FP32 products of L and K~ with blocks of at most cmax
// columns of Kuf (buffers of M x cmax floats).
void k_hutch_data(const float* Lf, const float* Kuu, const float* s, int M, int Mp, const float* Zs, const float* Xs,
                  int D, int B, const float* sf2, const float* m, bool precond, float* bufA, float* bufB,
                  float* bufC, int cmax, float* v, float* colq, double* red, cudaStream_t st);
// Tensor-core form of the P-free bound (hutchinson.cu): K~ in the operand
// precision; transposed operands (Np rows of Mp) of Kuf columns c0 .. c0+nc
// and of the probes; per-row q = 2|U_r|^2 - W_r . V_r; sums of row products.
template <class OutP> void k_kt_op(const float* Kuu, const float* s, int M, int Mp, OutP out, cudaStream_t st);
template <class OutP>
void k_kuf_t(const float* Zs, const float* Xs, int M, int Mp, int D, const float* sf2, int c0, int nc, int Np,
             OutP out, cudaStream_t st);
template <class OutP> void k_probes_t(const float* Z, int M, int Mp, int K, int Np, OutP out, cudaStream_t st);
template <class OutP>
void k_rowq(OutP U, OutP W, OutP V, int M, int Mp, int nc, float* q, double* dst, cudaStream_t st);
template <class OutP> void k_tdot(OutP X, OutP Y, int M, int Mp, int n, double* dst, cudaStream_t st);
// probit: E from red[RED_ELL], dsf2's data part from red[RED_SUMH], dnoise = 0.
// hutch_K > 0: tr(K~T) and tr(P Kuu) from the Hutchinson sums over hutch_K probes.
void k_terms_finalize(const double* red, const double* acc_ell, const float* sf2, const float* noise,
                      const float* ell, int M, int D, int B, double N, bool probit, int hutch_K, double* terms,
                      float* dsf2, float* dnoise, float* dell, int* errword, cudaStream_t st);
void k_predict_finalize(const float* colsum, const float* sf2, const float* noise, int Ns,
                        int include_noise, float* var, cudaStream_t st);
void k_adam(float* raw, float* cons, const float* grad, float* m1, float* m2, int* step,
            const float* hyper, const float* zbeta1, int M, int D, cudaStream_t st);
// Eq. (8) stopping rule from red[RED_NG_RESID], which it resets to 0 for the
// next iteration.
void k_ng_check(double* red, int M, double eps, int* done, int* iters, double* resid, int* errword,
                cudaStream_t st);
