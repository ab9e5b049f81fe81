// C-ABI of the R-SVGP library: handle, workspace, tile tables and the order
// of kernels for each entry point (see include/svgp.h for the contract).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "internal.h"

static unsigned long long g_launches = 0;
void svgp_note_launch() { __atomic_add_fetch(&g_launches, 1ull, __ATOMIC_RELAXED); }

namespace {

enum KRule { K_M0_END, K_N0_END, K_N0_M1, K_0_M1, K_0_N1, K_ALL };

std::vector<Tile> make_tiles(int Mp, int BM, int BN, int region, int rule) {
  std::vector<Tile> v;
  for (int m0 = 0; m0 < Mp; m0 += BM)
    for (int n0 = 0; n0 < Mp; n0 += BN) {
      if (region == REG_UPPER && m0 > n0 + BN - 1) continue;
      if (region == REG_LOWER && m0 + BM - 1 < n0) continue;
      Tile t{m0, n0, 0, Mp};
      int m1 = std::min(m0 + BM, Mp), n1 = std::min(n0 + BN, Mp);
      switch (rule) {
        case K_M0_END: t.k0 = m0; t.k1 = Mp; break;
        case K_N0_END: t.k0 = n0; t.k1 = Mp; break;
        case K_N0_M1: t.k0 = n0; t.k1 = m1; break;
        case K_0_M1: t.k0 = 0; t.k1 = m1; break;
        case K_0_N1: t.k0 = 0; t.k1 = n1; break;
        default: break;
      }
      if (t.k1 < t.k0) t.k1 = t.k0;
      v.push_back(t);
    }
  std::stable_sort(v.begin(), v.end(), [](const Tile& a, const Tile& b) { return (a.k1 - a.k0) > (b.k1 - b.k0); });
  return v;
}

}  // namespace

struct svgp_handle {
  svgp_config cfg;
  int M, Mp, D, Dp, Bmax;
  int mode;       // MODE_F32 / MODE_BF16 / MODE_SPLIT (svgp_prec)
  bool kuu3 = false;   // SVGP_BF16X3K: Kuu_lo holds a third plane for L^T K~
  cudaStream_t st;
  // second stream for Psi = Kuf Kuf^T, which depends only on the prologue:
  // forked from st after the prologue, joined before the first reader
  cudaStream_t st_aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool psi_pending = false;
  char err[512];
  // matrices
  float *Kuu_f, *Lf, *Pf, *Psi, *GKuu;
  void *Kuu_lo, *L_lo, *Lt_lo, *V, *S, *Y, *P_lo, *GP_lo;
  // vectors
  float *Zs, *Xs, *v, *w, *mu, *g, *Kg, *colsum, *rowacc_f, *rowacc_u, *dm_tmp;
  float* rowpart;   // partial row sets of the tensor-core W epilogue
  bool probit;      // Bernoulli-probit likelihood (else Gaussian)
  bool unprec;      // R-SVGP without the mean preconditioner (m = Kuu m~)
  GHRule gh;        // probit: Gauss-Hermite rule (weights divided by sqrt(pi))
  float* hn;        // probit: per-point h_n = dE_n/dsigma_n^2
  float* gapN;      // Prop. 3 gap: N = I - T K~ (FP32, Mp x Mp)
  float* hut;       // Hutchinson chains: three M x SVGP_HUTCH_KMAX buffers
  double *red, *acc_ell, *resid_tmp;
  int *errword, *done, *iters_tmp;
  GemmCtx gs, gt;   // SIMT and tensor-core tile tables
  // tensor-core schedule state per table: tiles, split threshold in force,
  // whether splitting is allowed, workspace slot range, item capacity
  std::vector<Tile> tc_tiles[TT_COUNT];
  int tc_kmin[TT_COUNT] = {0};
  bool may_split[TT_COUNT] = {false};
  int slot_base[TT_COUNT] = {0}, slot_cap[TT_COUNT] = {0}, item_cap[TT_COUNT] = {0};
  int rect_np[TT_COUNT] = {0};   // output columns of the tall-skinny table's current schedule
  KufTC kt;         // split coordinates for the tensor-core Kuf generator
  bool tc_kuf;      // Psi and W run on the tensor-core Kuf-producer kernels
  std::vector<void*> allocs;
  // instrumentation
  bool prof;
  std::vector<cudaEvent_t> ev;
  std::vector<int> rec_kind;
};

namespace {

svgp_status fail(svgp_handle* h, svgp_status s, const char* msg) {
  if (h) snprintf(h->err, sizeof(h->err), "%s", msg);
  return s;
}

svgp_status check_launch(svgp_handle* h, const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    snprintf(h->err, sizeof(h->err), "%s: %s", where, cudaGetErrorString(e));
    return SVGP_ERR_CUDA;
  }
  return SVGP_OK;
}

template <class T>
bool dalloc(svgp_handle* h, T** p, size_t bytes) {
  void* q = nullptr;
  if (cudaMalloc(&q, bytes) != cudaSuccess) return false;
  cudaMemset(q, 0, bytes);
  h->allocs.push_back(q);
  *p = reinterpret_cast<T*>(q);
  return true;
}

bool upload_tiles(svgp_handle* h, const std::vector<Tile>& v, Tile** out, int* n) {
  if (!dalloc(h, out, sizeof(Tile) * std::max<size_t>(v.size(), 1))) return false;
  cudaMemcpy(*out, v.data(), sizeof(Tile) * v.size(), cudaMemcpyHostToDevice);
  *n = (int)v.size();
  return true;
}

// Persistent-kernel schedule.  Cost model of a work item in cycles: k-blocks x
// 750 (the measured mainloop cost per 64-deep k-block) plus its epilogue (5000
// for a whole or owner item, 2000 more for the owner's read of the partial,
// 1500 for a producer's partial store).
long long item_cost(const TcTile& t) {
  const long long k = (long long)(t.k1 - t.k0) / 64 * 750;
  return k + (t.role == TC_PRODUCER ? 1500 : t.role == TC_OWNER ? 7000 : 5000);
}

// Longest-processing-time-first assignment of the items to min(#items, nsm)
// CTAs; within a CTA producer chunks come first (they never wait, so every
// owner's producer finishes whatever the owners do), then the rest by
// decreasing cost.  Returns the items grouped by CTA (off[c] .. off[c + 1]
// are CTA c's) and the modelled makespan.
std::vector<TcTile> lpt_schedule(std::vector<TcTile> v, int nsm, std::vector<int>& off, long long* makespan) {
  std::stable_sort(v.begin(), v.end(), [](const TcTile& a, const TcTile& b) { return item_cost(a) > item_cost(b); });
  const int G = std::max(1, std::min((int)v.size(), nsm));
  std::vector<std::vector<TcTile>> per(G);
  std::vector<long long> load(G, 0);
  for (const TcTile& t : v) {
    int c = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    per[c].push_back(t);
    load[c] += item_cost(t);
  }
  std::vector<TcTile> out;
  off.assign(1, 0);
  for (int c = 0; c < G; ++c) {
    std::stable_partition(per[c].begin(), per[c].end(), [](const TcTile& t) { return t.role == TC_PRODUCER; });
    out.insert(out.end(), per[c].begin(), per[c].end());
    off.push_back((int)out.size());
  }
  if (makespan) *makespan = *std::max_element(load.begin(), load.end());
  return out;
}

// Split-K plan of a tile table: tiles of at least kmin k-blocks become a
// producer and an owner chunk (K boundary at a 64 multiple, slots from
// *slot); kmin = 0 splits nothing.
std::vector<TcTile> split_items(const std::vector<Tile>& v, int kmin, int* slot) {
  std::vector<TcTile> out;
  for (const Tile& t : v) {
    const int nk = (t.k1 - t.k0) / 64;
    if (kmin > 0 && nk >= kmin) {
      const int kmid = t.k0 + (nk / 2) * 64;
      out.push_back(TcTile{t.m0, t.n0, t.k0, kmid, TC_PRODUCER, *slot});
      out.push_back(TcTile{t.m0, t.n0, kmid, t.k1, TC_OWNER, *slot});
      ++*slot;
    } else {
      out.push_back(TcTile{t.m0, t.n0, t.k0, t.k1, TC_WHOLE, 0});
    }
  }
  return out;
}

// Split thresholds a table may take: 0 (no split) or a fraction of its
// longest tile's k-blocks (1, 7/8, 3/4, 5/8, 1/2, 3/8), at least 2.
std::vector<int> split_candidates(const std::vector<Tile>& v) {
  int maxnk = 0;
  for (const Tile& t : v) maxnk = std::max(maxnk, (t.k1 - t.k0) / 64);
  std::vector<int> c{0};
  for (int q : {8, 7, 6, 5, 4, 3}) {
    const int k = (maxnk * q + 7) / 8;
    if (k >= 2 && std::find(c.begin(), c.end(), k) == c.end()) c.push_back(k);
  }
  return c;
}

// The candidate with the smallest modelled makespan (ties within 3 %: fewer splits).
int model_kmin(const std::vector<Tile>& v, int nsm) {
  int best = 0;
  long long best_ms = 0;
  for (int kmin : split_candidates(v)) {
    int tmp = 0;
    std::vector<int> o;
    long long ms = 0;
    lpt_schedule(split_items(v, kmin, &tmp), nsm, o, &ms);
    if (kmin == 0 || ms < best_ms * 97 / 100) { best = kmin; best_ms = ms; }
  }
  return best;
}

// Tiles that some candidate threshold would split (the slots a table may need).
int split_capacity(const std::vector<Tile>& v) {
  const std::vector<int> c = split_candidates(v);
  int kmin = 0;
  for (int k : c)
    if (k > 0 && (kmin == 0 || k < kmin)) kmin = k;
  int n = 0;
  for (const Tile& t : v) n += (kmin > 0 && (t.k1 - t.k0) / 64 >= kmin) ? 1 : 0;
  return n;
}

// Tensor-core schedule of table `tab` with split threshold kmin (0: whole
// tiles), into the table's preallocated item and offset buffers; slots from
// the table's own range.  Host-synchronous (configuration time only).
bool schedule_table(svgp_handle* h, int tab, int kmin) {
  GemmCtx& g = h->gt;
  int slot = h->slot_base[tab];
  std::vector<int> off;
  std::vector<TcTile> s = lpt_schedule(split_items(h->tc_tiles[tab], kmin, &slot), tc_num_sms(), off, nullptr);
  if (slot - h->slot_base[tab] > h->slot_cap[tab] || s.size() > (size_t)h->item_cap[tab]) return false;
  if (cudaMemcpy(g.tct[tab], s.data(), sizeof(TcTile) * s.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(g.toff[tab], off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return false;
  g.nt[tab] = (int)s.size();
  g.ncta[tab] = (int)off.size() - 1;
  h->tc_kmin[tab] = kmin;
  return true;
}

// Schedule of a tall-skinny table for output columns [0, Np) (whole tiles).
// Host-synchronous when Np changes: the handle's streams are drained before
// the device tables are rewritten.
bool rect_schedule(svgp_handle* h, int tab, int Np) {
  if (h->rect_np[tab] == Np) return true;
  if (cudaStreamSynchronize(h->st) != cudaSuccess || cudaStreamSynchronize(h->st_aux) != cudaSuccess) return false;
  std::vector<Tile> v;
  for (const Tile& t : h->tc_tiles[tab])
    if (t.n0 < Np) v.push_back(t);
  // long K ranges over few output tiles: split where the cost model gains,
  // within the workspace slots the three tall-skinny tables share (they run
  // one after another on one stream)
  const int kmin = (Np / 128) * (h->Mp / 128) <= h->slot_cap[tab] ? model_kmin(v, tc_num_sms()) : 0;
  int slot = h->slot_base[tab];
  std::vector<int> off;
  GemmCtx& g = h->gt;
  std::vector<TcTile> s = lpt_schedule(split_items(v, kmin, &slot), tc_num_sms(), off, nullptr);
  if (s.size() > (size_t)h->item_cap[tab] || slot - h->slot_base[tab] > h->slot_cap[tab]) return false;
  if (cudaMemcpy(g.tct[tab], s.data(), sizeof(TcTile) * s.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(g.toff[tab], off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return false;
  g.nt[tab] = (int)s.size();
  g.ncta[tab] = (int)off.size() - 1;
  h->rect_np[tab] = Np;
  return true;
}

bool build_ctx(svgp_handle* h, GemmCtx& g, int BM, int BN, bool sched) {
  int Mp = h->Mp;
  g.Mp = Mp;
  g.st = h->st;
  g.err = h->errword;
  g.split = h->mode == 2;
  const std::vector<Tile> tabs[TT_COUNT] = {
      make_tiles(Mp, BM, BN, REG_FULL, K_M0_END),  make_tiles(Mp, BM, BN, REG_UPPER, K_N0_END),
      make_tiles(Mp, BM, BN, REG_LOWER, K_N0_M1),  make_tiles(Mp, BM, BN, REG_FULL, K_0_M1),
      make_tiles(Mp, BM, BN, REG_LOWER, K_0_N1),   make_tiles(Mp, BM, BN, REG_UPPER, K_ALL),
      make_tiles(Mp, BM, BN, REG_FULL, K_ALL),     make_tiles(Mp, BM, BN, REG_FULL, K_0_M1),
      make_tiles(Mp, BM, BN, REG_FULL, K_M0_END),  make_tiles(Mp, BM, BN, REG_FULL, K_ALL)};
  if (!sched) {
    for (int t = 0; t < TT_COUNT; ++t)
      if (!upload_tiles(h, tabs[t], &g.tt[t], &g.nt[t])) return false;
    return true;
  }
  // tensor-core schedules: the triangular tables (symmetric and lower
  // outputs) may split long tiles, with the threshold of the cost model
  // until svgp_set_split chooses another
  int slot = 0;
  // the tall-skinny tables share one slot range: split schedules for up to
  // four output column tiles (Np <= 512)
  const int rect_cap = (Mp / 128) * std::min(Mp / 128, 4);
  for (int t = 0; t < TT_COUNT; ++t) {
    if (t == TT_PSI) {
      if (!upload_tiles(h, tabs[t], &g.tt[t], &g.nt[t])) return false;
      continue;
    }
    h->tc_tiles[t] = tabs[t];
    h->may_split[t] = t == TT_SYM_IN || t == TT_LUPD || t == TT_OUT;
    h->slot_base[t] = slot;
    h->slot_cap[t] = h->may_split[t] ? split_capacity(tabs[t]) : (t >= TT_RL ? rect_cap : 0);
    h->item_cap[t] = (int)tabs[t].size() + h->slot_cap[t];
    if (t < TT_RL || t == TT_COUNT - 1) slot += h->slot_cap[t];
    if (!dalloc(h, &g.tct[t], sizeof(TcTile) * std::max(h->item_cap[t], 1)) ||
        !dalloc(h, &g.toff[t], sizeof(int) * (size_t)(tc_num_sms() + 1)))
      return false;
  }
  g.nslot = slot;
  if (slot > 0 && !(dalloc(h, &g.kpart, sizeof(float) * 128 * 128 * (size_t)slot) &&
                    dalloc(h, &g.kflag, sizeof(int) * 2 * (size_t)slot)))
    return false;
  for (int t = 0; t < TT_COUNT; ++t) {
    if (t == TT_PSI || t >= TT_RL) continue;       // the tall-skinny tables are scheduled per call
    const int kmin = h->may_split[t] ? model_kmin(tabs[t], tc_num_sms()) : 0;
    if (!schedule_table(h, t, kmin)) return false;
  }
  return true;
}

bool valid_params(const svgp_handle* h, const svgp_params* p) {
  return p && p->Z && p->ell && p->sf2 && (p->noise || h->probit) && p->m && p->s && p->L;
}

// Brackets one launch with timing events while profiling is enabled.
// Inside a stream capture the records are external (event-record nodes of
// the graph, re-recorded at every replay); outside, plain records.
void prof_record(cudaEvent_t e, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cs);
  if (cs == cudaStreamCaptureStatusActive) cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
  else cudaEventRecord(e, st);
}

struct ProfScope {
  svgp_handle* h; int idx;
  ProfScope(svgp_handle* hh, int kind) : h(hh), idx(-1) {
    if (!h->prof) return;
    int n = (int)h->rec_kind.size();
    if (2 * n + 1 >= (int)h->ev.size()) return;
    idx = n;
    h->rec_kind.push_back(kind);
    prof_record(h->ev[2 * n], h->st);
  }
  ~ProfScope() {
    if (idx >= 0) prof_record(h->ev[2 * idx + 1], h->st);
  }
};

// ---------------------------------------------------------------------------
// Precision dispatch of the M x M GEMM chain.
// ---------------------------------------------------------------------------
enum Mode { MODE_F32 = 0, MODE_BF16 = 1, MODE_SPLIT = 2 };

float* F(void* p) { return reinterpret_cast<float*>(p); }
bf16* H(void* p) { return reinterpret_cast<bf16*>(p); }
SplitPtr SP(const svgp_handle* h, void* p) {
  return SplitPtr{reinterpret_cast<bf16*>(p), reinterpret_cast<bf16*>(p) + (size_t)h->Mp * h->Mp};
}
Split3Ptr SP3(const svgp_handle* h, void* p) {
  bf16* b = reinterpret_cast<bf16*>(p);
  const size_t MM = (size_t)h->Mp * h->Mp;
  return Split3Ptr{b, b + MM, b + 2 * MM};
}

// Calls simt_gemm / tc_gemm with the functor built for the handle's mode.
#define DISPATCH(h, tab, A, B, MAKE)                                                         \
  do {                                                                                       \
    if ((h)->mode == MODE_F32) simt_gemm((h)->gs, tab, F(A), F(B), MAKE(float*, F));         \
    else if ((h)->mode == MODE_BF16) tc_gemm((h)->gt, tab, H(A), H(B), MAKE(bf16*, H));      \
    else tc_gemm((h)->gt, tab, H(A), H(B), MAKE(SplitPtr, SPH));                             \
  } while (0)

void run_vt(svgp_handle* h, void* B, const float* s, const int* skip) {
  ProfScope ps(h, SVGP_PROF_VT);
  auto SPH = [h](void* p) { return SP(h, p); };
#define MK(T, CV) EpiVt<T>{CV(h->V), h->Mp, h->Lf, s, h->M, skip}
  if (h->kuu3 && B == h->Kuu_lo)   // K~ with its third plane: five MMAs per product
    tc_gemm(h->gt, TT_VT, H(h->Lt_lo), H(B), MK(SplitPtr, SPH), H(B) + 2 * (size_t)h->Mp * h->Mp);
  else
    DISPATCH(h, TT_VT, h->Lt_lo, B, MK);
#undef MK
}

template <int MODE>
void run_sym(svgp_handle* h, const int* skip) {
  ProfScope ps(h, SVGP_PROF_SYM);
  auto SPH = [h](void* p) { return SP(h, p); };
#define MK(T, CV) EpiSym<T, MODE>{CV(h->S), h->Mp, h->M, h->red, skip}
  DISPATCH(h, TT_SYM_IN, h->V, h->Lt_lo, MK);
#undef MK
}

void run_ls(svgp_handle* h) {  // Y = L S
  ProfScope ps(h, SVGP_PROF_LS);
  auto SPH = [h](void* p) { return SP(h, p); };
#define MK(T, CV) EpiStore<T>{CV(h->Y), h->Mp, nullptr}
  DISPATCH(h, TT_LS, h->L_lo, h->S, MK);
#undef MK
}

void run_p(svgp_handle* h, const float* s, const float* Psi) {  // P = Y L^T
  ProfScope ps(h, SVGP_PROF_OUT);
  auto SPH = [h](void* p) { return SP(h, p); };
#define MK(T, CV) EpiP<T>{h->Pf, CV(h->P_lo), h->Mp, h->M, s, Psi, h->red}
  DISPATCH(h, TT_OUT, h->Y, h->L_lo, MK);
#undef MK
}

void run_gk(svgp_handle* h, const float* s, float* ds) {  // G_K~ = -Y L^T
  ProfScope ps(h, SVGP_PROF_OUT);
  EpiGK e{h->GKuu, h->Mp, h->M, h->Pf, h->v, s, ds};
  if (h->mode == MODE_F32) simt_gemm(h->gs, TT_OUT, F(h->Y), F(h->L_lo), e);
  else tc_gemm(h->gt, TT_OUT, H(h->Y), H(h->L_lo), e);
}

void run_lupd(svgp_handle* h, float* L_inout, const float* gamma) {  // L <- L - gamma L Phi
  ProfScope ps(h, SVGP_PROF_LUPD);
  EpiLupd e{h->Lf, h->Mp, L_inout, h->M, gamma, h->done};
  if (h->mode == MODE_F32) simt_gemm(h->gs, TT_LUPD, F(h->L_lo), F(h->S), e);
  else tc_gemm(h->gt, TT_LUPD, H(h->L_lo), H(h->S), e);
}

// Psi = Kuf Kuf^T, or Kuf diag(|hw|) Kuf^T when hw != null (the tensor-core
// path then reads the weighted k-role vectors kt.XKh, prepared from hw).
void run_psi(svgp_handle* h, const svgp_params* p, int B, const float* hw) {
  ProfScope ps(h, SVGP_PROF_PSI);
  KufGen kg{h->Zs, h->Xs, h->D, h->M, B, p->sf2};
  EpiPsi e{h->Psi, h->Mp};
  if (!(h->tc_kuf && tc_psi(h->gt, kg, h->kt, hw ? h->kt.XKh : h->kt.XK, B, e))) simt_psi(h->gs, kg, B, e, hw);
}

// Psi of the Gaussian bound on the second stream (it needs only the
// prologue's coordinates and Kuf operands): the products that follow on st
// do not wait for it until join_psi, so Psi fills the SMs their tails leave.
// Runs f's launches on the second stream after everything issued so far on
// st; join_aux makes st wait for them.
template <class F>
void on_aux(svgp_handle* h, F&& f) {
  cudaEventRecord(h->ev_fork, h->st);
  cudaStreamWaitEvent(h->st_aux, h->ev_fork, 0);
  cudaStream_t main = h->st;
  h->st = h->gs.st = h->gt.st = h->st_aux;
  f();
  h->st = h->gs.st = h->gt.st = main;
  cudaEventRecord(h->ev_join, h->st_aux);
}

void join_aux(svgp_handle* h) { cudaStreamWaitEvent(h->st, h->ev_join, 0); }

void fork_psi(svgp_handle* h, const svgp_params* p, int B) {
  if (h->psi_pending || h->probit) return;
  on_aux(h, [&] { run_psi(h, p, B, nullptr); });
  h->psi_pending = true;
}

void join_psi(svgp_handle* h) {
  if (!h->psi_pending) return;
  join_aux(h);
  h->psi_pending = false;
}

// Returns the number of partial row sets the tensor-core kernel wrote (0 when
// the SIMT kernel accumulated into we.rowacc, or in variance mode).
int run_w(svgp_handle* h, const WEpi& we) {
  ProfScope ps(h, SVGP_PROF_W);
  const int n = h->tc_kuf ? tc_w(h->gt, H(h->P_lo), h->kt, we, h->rowpart) : -1;
  if (n >= 0) return n;
  simt_w(h->gs, h->Pf, we);
  return 0;
}

// FP32 and operand copies of L (and L^T); adds sum_i log|L_ii| to *logdet
// when logdet != null.
void prep_L(svgp_handle* h, const float* Lin, double* logdet) {
  if (h->mode == MODE_F32) k_prep_L(Lin, h->M, h->Mp, h->Lf, F(h->L_lo), F(h->Lt_lo), logdet, h->st);
  else if (h->mode == MODE_BF16) k_prep_L(Lin, h->M, h->Mp, h->Lf, H(h->L_lo), H(h->Lt_lo), logdet, h->st);
  else k_prep_L(Lin, h->M, h->Mp, h->Lf, SP(h, h->L_lo), SP(h, h->Lt_lo), logdet, h->st);
}

// Common prologue: scaled coordinates, Kuu, L copies, log-det of L (unless
// logdet_L is false); zero sums.  One launch zeroes every accumulator the
// forward and backward passes that follow add into (mu and Kuf g of the
// tensor-core gemvs, the row sums of the chain rules), and the NG loop's
// flag and counter when given.
void prologue(svgp_handle* h, const svgp_params* p, const float* X, int B, const float* Lin, bool logdet_L = true,
              int* ng_done = nullptr, int* ng_iters = nullptr) {
  cudaStream_t st = h->st;
  const size_t rows = sizeof(float) * (size_t)h->Mp * (2 * h->D + 1);
  const ZeroRange zr[8] = {{h->red, sizeof(double) * RED_COUNT}, {h->acc_ell, sizeof(double) * SVGP_MAXD},
                           {X ? h->mu : nullptr, sizeof(float) * (size_t)B}, {h->Kg, sizeof(float) * (size_t)h->Mp},
                           {h->rowacc_f, rows}, {h->rowacc_u, rows},
                           {ng_done, sizeof(int)}, {ng_iters, sizeof(int)}};
  k_zero_n(st, zr, 8);
  k_prep_coords(p->Z, X, p->ell, h->M, h->Mp, X ? B : 0, h->D, h->Zs, h->Xs, st, p->s, h->red + RED_LOGS);
  if (h->tc_kuf) k_kuf_prep(h->Zs, X ? h->Xs : nullptr, h->M, h->Mp, X ? B : 0, (B + 127) / 128 * 128, h->D, p->sf2, h->kt, st);
  if (h->mode == MODE_F32) k_kuu(h->Zs, h->M, h->Mp, h->D, p->sf2, h->Kuu_f, (float*)nullptr, false, st);
  else if (h->mode == MODE_BF16) k_kuu(h->Zs, h->M, h->Mp, h->D, p->sf2, h->Kuu_f, H(h->Kuu_lo), true, st);
  else if (h->kuu3) k_kuu(h->Zs, h->M, h->Mp, h->D, p->sf2, h->Kuu_f, SP3(h, h->Kuu_lo), true, st);
  else k_kuu(h->Zs, h->M, h->Mp, h->D, p->sf2, h->Kuu_f, SP(h, h->Kuu_lo), true, st);
  prep_L(h, Lin, logdet_L ? h->red + RED_LOGDETL : nullptr);
}

// Forward pass of Eq. (7) up to the per-point likelihood terms.  Gaussian:
// sum_n sigma_n^2 through <P, Psi> (psi = true builds Psi); probit: sigma_n^2
// per point from the column sums of Kuf o (P Kuf), then the quadrature.
void forward(svgp_handle* h, const svgp_params* p, const svgp_batch* b, bool psi) {
  cudaStream_t st = h->st;
  psi = psi && !h->probit;
  if (psi) fork_psi(h, p, b->B);         // Psi = Kuf Kuf^T (Kuf generated on chip), second stream
  run_vt(h, h->Kuu_lo, p->s, nullptr);   // Vt = L^T K~
  run_sym<1>(h, nullptr);                // A1 = L^T K~ L ; S = 2I - A1 ; tr, Frobenius
  run_ls(h);                             // Y = L (2I - A1)
  if (psi) join_psi(h);
  run_p(h, p->s, psi ? h->Psi : nullptr);  // P = Y L^T ; sum s_i P_ii ; <P, Psi>
  if (h->unprec) cudaMemcpyAsync(h->v, p->m, sizeof(float) * h->M, cudaMemcpyDeviceToDevice, st);  // v = m
  else k_gemv(h->Pf, h->Mp, h->M, p->m, 1.f, nullptr, 0.f, h->v, nullptr, nullptr, st);     // v = P m
  k_gemv(h->Kuu_f, h->Mp, h->M, h->v, 1.f, nullptr, 0.f, h->w, h->v, h->red + RED_QUAD, st);  // w = Kuu v
  if (b) {
    if (!(h->tc_kuf && tc_kuf_gemv(h->kt.XR, b->B, h->kt.ZK, h->M, h->v, h->mu, true, h->errword, st)))
      k_mu(h->Zs, h->Xs, h->M, b->B, h->D, p->sf2, h->v, h->mu, st);                        // mu = Kfu v
    if (h->probit) {
      k_zero(st, h->colsum, sizeof(float) * b->B);
      WEpi wv{KufGen{h->Zs, h->Xs, h->D, h->M, b->B, p->sf2}, nullptr, nullptr, nullptr, nullptr, 0.f, nullptr,
              h->colsum};
      run_w(h, wv);                                                                       // k_n^T P k_n
      k_pointwise_probit(b->y, h->mu, h->colsum, p->sf2, b->B, h->gh, h->g, h->hn, h->red, st);
    } else {
      k_pointwise_gauss(b->y, h->mu, p->noise, b->B, h->g, h->red, st);
    }
  }
}

svgp_status validate_batch(svgp_handle* h, const svgp_batch* b) {
  if (!b || !b->X || !b->y) return fail(h, SVGP_ERR_INVALID_ARG, "batch: null pointer");
  if (b->B < 1 || b->B > h->Bmax) return fail(h, SVGP_ERR_INVALID_ARG, "batch: B out of [1, B_max]");
  if (!(b->N > 0)) return fail(h, SVGP_ERR_INVALID_ARG, "batch: N must be > 0");
  return SVGP_OK;
}

bool valid_grads(const svgp_grads* gr) {
  return gr && gr->dZ && gr->dell && gr->dsf2 && gr->dnoise && gr->dm && gr->ds;
}
// Bound and gradient after the prologue: forward pass, then the backward
// pass with T fixed (Section 3.1).
void backward_tail(svgp_handle* h, const svgp_params* p, const svgp_batch* b, double* terms_dev, const svgp_grads* gr) {
  cudaStream_t st = h->st;
  const int M = h->M, Mp = h->Mp;
  const float c = (float)(b->N / b->B);
  forward(h, p, b, true);
  if (h->probit) {                                                                      // Kuf diag(|h|) Kuf^T
    if (h->tc_kuf) k_kuf_prep_weighted(h->Xs, b->B, (b->B + 127) / 128 * 128, h->D, p->sf2, h->hn, h->kt.XKh, st);
    run_psi(h, p, b->B, h->hn);
  }
  if (!(h->tc_kuf && tc_kuf_gemv(h->kt.ZR, M, h->kt.XK, b->B, h->g, h->Kg, true, h->errword, st)))
    k_kg(h->Zs, h->Xs, M, Mp, b->B, h->D, p->sf2, h->g, h->Kg, st);                    // Kuf g
  // W = P Kuf with the data part of the chain rule, and dm~, need only the
  // forward pass and Kuf g: on the second stream, beside the G_Kuu chain;
  // joined before the gradient finalize
  const float* nz0 = h->probit ? nullptr : p->noise;
  WEpi we{KufGen{h->Zs, h->Xs, h->D, M, b->B, p->sf2}, h->v, h->g, h->probit ? h->hn : nullptr, nz0, c,
          h->rowacc_f, nullptr};
  int nparts = 0;
  on_aux(h, [&] {
    nparts = run_w(h, we);                                                                // data part of dZ, dell, dsf2
    if (h->unprec) k_axpy(h->Kg, c, h->w, -1.0f / c, gr->dm, M, h->st);                // dm = c Kg - w
    else k_gemv(h->Pf, Mp, M, h->Kg, c, h->w, -1.0f / c, gr->dm, nullptr, nullptr, h->st); // dm = P (c Kg - w)
  });
  const float* nz = h->probit ? nullptr : p->noise;
  const float* mt = h->unprec ? nullptr : p->m;
  if (h->mode == MODE_F32) k_gp_assemble(h->Kuu_f, h->Psi, h->Kg, mt, h->w, nz, c, M, Mp, F(h->GP_lo), st);
  else if (h->mode == MODE_BF16) k_gp_assemble(h->Kuu_f, h->Psi, h->Kg, mt, h->w, nz, c, M, Mp, H(h->GP_lo), st);
  else k_gp_assemble(h->Kuu_f, h->Psi, h->Kg, mt, h->w, nz, c, M, Mp, SP(h, h->GP_lo), st);
  run_vt(h, h->GP_lo, nullptr, nullptr); // X1t = L^T G_P
  run_sym<2>(h, nullptr);                // S = L^T G_P L + I/2
  run_ls(h);                             // Y = L S
  run_gk(h, p->s, gr->ds);               // G_K~ = -Y L^T -> G_Kuu, ds
  k_kuu_bwd(h->GKuu, h->Kuu_f, h->Zs, M, Mp, h->D, h->rowacc_u, h->red, st);          // Kuu part
  join_aux(h);                                                                         // W and dm done
  k_grad_finalize(h->rowacc_f, h->rowacc_u, h->rowpart, nparts, Mp, p->ell, M, h->D, gr->dZ, h->acc_ell, h->red,
                  st);
  k_terms_finalize(h->red, h->acc_ell, p->sf2, p->noise, p->ell, M, h->D, b->B, b->N, h->probit, 0, terms_dev,
                   gr->dsf2, gr->dnoise, gr->dell, h->errword, st);
}

// NG iterations of Prop. 1 on L_inout after the prologue (K~ and the L copies
// current); the L copies are refreshed between iterations, not after the last.
void ng_loop(svgp_handle* h, const svgp_params* p, float* L_inout, const float* gamma_dev, int max_iters, double eps,
             int* iters, double* resid, bool zeroed = false) {
  cudaStream_t st = h->st;
  // red[RED_NG_RESID] starts at 0 (prologue) and ng_check resets it after reading;
  // done and iters start at 0 (here, or in the prologue when zeroed)
  if (!zeroed) k_zero(st, h->done, sizeof(int), iters, sizeof(int));
  for (int t = 0; t < max_iters; ++t) {
    run_vt(h, h->Kuu_lo, p->s, h->done);         // Vt = L^T K~ (skipped once converged)
    run_sym<0>(h, h->done);                      // A, Phi^T, ||A - I||^2
    k_ng_check(h->red, h->M, eps, h->done, iters, resid, h->errword, st);   // Eq. (8) stopping rule
    run_lupd(h, L_inout, gamma_dev + t);         // L <- L - gamma L Phi  (Prop. 1)
    if (t + 1 < max_iters) prep_L(h, L_inout, nullptr);
  }
}

// Prop. 3 gap for the current L (FP32 copy h->Lf) and the batch's Psi:
// red[RED_GAPDOT] += <N N^T, Psi> with N = I - T K~, T = L L^T, K~ in FP32
// (h->GKuu) -- three FP32 SIMT products: T = L L^T (into h->Pf), N, and
// N N^T reduced against Psi.  Skipped while *skip != 0.
void gap_compute(svgp_handle* h, const int* skip) {
  const int M = h->M, Mp = h->Mp;
  simt_gemm(h->gs, TT_LS, h->Lf, h->Lf, EpiStore<float*>{h->Pf, Mp, skip});
  simt_gemm(h->gs, TT_FULL, h->Pf, h->GKuu, EpiIminus{h->gapN, Mp, M, skip});
  simt_gemm(h->gs, TT_FULL, h->gapN, h->gapN, EpiDotPsi{h->Psi, Mp, M, h->red + RED_GAPDOT, skip});
}

// Tall-skinny product of the P-free bound on the tensor cores: out^T =
// (A X)^T over output columns [0, Np), with X given as X^T (Np rows of Mp).
template <class OutP>
bool rect_product(svgp_handle* h, int tab, const bf16* A, const bf16* Bt, OutP outT, int Np) {
  if (!rect_schedule(h, tab, Np)) return false;
  return tc_gemm(h->gt, tab, A, Bt, EpiStoreT<OutP>{outT, h->Mp});
}

// The P-free bound's products (Section 3.4) on the tensor cores in the
// handle's operand precision: k_n^T P k_n = 2 |L^T k_n|^2 - w^T K~ w with
// w = T k_n for blocks of up to Mp points, and the three probe chains of
// the traces.  Factors are kept transposed in the handle's idle M x M operand
// buffers (Y, V, S, P_lo, GP_lo).  One column count Np for every product of
// the call (the larger of the point block and the probe block), so that the
// schedules are rewritten only when B or K changes between calls.
template <class OutP, class Conv>
bool hutch_tc(svgp_handle* h, const svgp_params* p, const svgp_batch* b, const float* probes, int K, Conv cv) {
  cudaStream_t st = h->st;
  const int M = h->M, Mp = h->Mp;
  OutP Kt = cv(h->GP_lo), Xt = cv(h->S), Ut = cv(h->Y), Wt = cv(h->V), Zt = cv(h->P_lo);
  const bf16* Lh = H(h->L_lo);
  const bf16* Lth = H(h->Lt_lo);
  const bf16* Kuh = H(h->Kuu_lo);
  const bf16* Kth = H(h->GP_lo);
  auto hi = [](void* q) { return reinterpret_cast<const bf16*>(q); };
  k_kt_op(h->Kuu_f, p->s, M, Mp, Kt, st);
  const int Np = std::max((std::min(Mp, b->B) + 127) / 128, (K + 127) / 128) * 128;
  for (int c0 = 0; c0 < b->B; c0 += Mp) {
    const int nc = std::min(Mp, b->B - c0);
    k_kuf_t(h->Zs, h->Xs, M, Mp, h->D, p->sf2, c0, nc, Np, Xt, st);
    if (!rect_product(h, TT_RLT, Lth, hi(h->S), Ut, Np) ||          // u = L^T k
        !rect_product(h, TT_RL, Lh, hi(h->Y), Wt, Np) ||            // w = L u
        !rect_product(h, TT_RF, Kth, hi(h->V), Zt, Np))             // K~ w
      return false;
    k_rowq(Ut, Wt, Zt, M, Mp, nc, h->colsum + c0, h->red + RED_PPSI, st);
  }
  // traces: y = L z, <y, K~ y>;  c = T Kuu z, <z, c>;  f = T K~ c, <z, f>
  OutP Pt = cv(h->S), Y = cv(h->Y), V = cv(h->V), E = cv(h->P_lo);
  k_probes_t(probes, M, Mp, K, Np, Pt, st);
  if (!rect_product(h, TT_RL, Lh, hi(h->S), Y, Np) || !rect_product(h, TT_RF, Kth, hi(h->Y), V, Np))
    return false;
  k_tdot(Y, V, M, Mp, K, h->red + RED_HKT, st);
  if (!rect_product(h, TT_RF, Kuh, hi(h->S), Y, Np) || !rect_product(h, TT_RLT, Lth, hi(h->Y), V, Np) ||
      !rect_product(h, TT_RL, Lh, hi(h->V), Y, Np))
    return false;
  k_tdot(Pt, Y, M, Mp, K, h->red + RED_HW1, st);
  if (!rect_product(h, TT_RF, Kth, hi(h->Y), V, Np) || !rect_product(h, TT_RLT, Lth, hi(h->V), E, Np) ||
      !rect_product(h, TT_RL, Lh, hi(h->P_lo), V, Np))
    return false;
  k_tdot(Pt, V, M, Mp, K, h->red + RED_HX4, st);
  return true;
}

bool valid_ng_args(const svgp_params* p, const float* L_inout, const float* gamma_dev, int max_iters) {
  return p && p->Z && p->ell && p->sf2 && p->s && L_inout && gamma_dev && max_iters >= 0 && max_iters <= 100000;
}


}  // namespace

extern "C" {

const char* svgp_status_string(int s) {
  switch (s) {
    case SVGP_OK: return "ok";
    case SVGP_ERR_INVALID_ARG: return "invalid argument";
    case SVGP_ERR_CUDA: return "CUDA error";
    case SVGP_ERR_OOM: return "out of device memory";
    case SVGP_ERR_NONFINITE: return "non-finite value on device";
    case SVGP_ERR_NOT_CONVERGED: return "not converged";
    case SVGP_ERR_TIMEOUT: return "device wait timed out";
    case SVGP_ERR_UNSUPPORTED: return "unsupported";
    default: return "unknown status";
  }
}

int svgp_has_tensor_cores(void) { return tc_available() ? 1 : 0; }

svgp_status svgp_gauss_hermite(int n, double* nodes, double* weights) {
  return gauss_hermite_rule(n, nodes, weights) ? SVGP_OK : SVGP_ERR_INVALID_ARG;
}

svgp_status svgp_create(const svgp_config* cfg, svgp_handle** out) {
  if (!cfg || !out) return SVGP_ERR_INVALID_ARG;
  *out = nullptr;
  if (cfg->M < 1 || cfg->M > 8192 || cfg->D < 1 || cfg->D > SVGP_MAXD || cfg->B_max < 1 ||
      cfg->B_max > (1 << 22))
    return SVGP_ERR_INVALID_ARG;
  if (cfg->lik != SVGP_LIK_GAUSSIAN && cfg->lik != SVGP_LIK_BERNOULLI_PROBIT) return SVGP_ERR_INVALID_ARG;
  if (cfg->lik == SVGP_LIK_BERNOULLI_PROBIT && (cfg->gh_points < 0 || cfg->gh_points > GH_MAX))
    return SVGP_ERR_INVALID_ARG;
  if (cfg->prec != SVGP_FP32 && cfg->prec != SVGP_BF16 && cfg->prec != SVGP_BF16X3 && cfg->prec != SVGP_BF16X3K)
    return SVGP_ERR_INVALID_ARG;
  if (cfg->prec != SVGP_FP32 && !tc_available()) return SVGP_ERR_UNSUPPORTED;
  svgp_handle* h = new svgp_handle();
  h->cfg = *cfg;
  h->M = cfg->M;
  h->Mp = (cfg->M + 127) / 128 * 128;
  h->D = cfg->D;
  h->Dp = (cfg->D + 3) & ~3;
  h->Bmax = cfg->B_max;
  h->kuu3 = cfg->prec == SVGP_BF16X3K;
  h->mode = h->kuu3 ? MODE_SPLIT : cfg->prec;   // svgp_prec values 0..2 coincide with MODE_*
  h->st = (cudaStream_t)cfg->cuda_stream;
  if (cudaStreamCreateWithFlags(&h->st_aux, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    svgp_destroy(h);
    return SVGP_ERR_CUDA;
  }
  h->err[0] = 0;
  h->prof = false;
  h->probit = cfg->lik == SVGP_LIK_BERNOULLI_PROBIT;
  h->unprec = cfg->unpreconditioned != 0;
  h->gh.n = 0;
  h->hn = nullptr;
  h->kt.XKh = nullptr;
  if (h->probit) {
    h->gh.n = cfg->gh_points > 0 ? cfg->gh_points : 20;
    double t[64], w[64];
    if (!gauss_hermite_rule(h->gh.n, t, w)) {
      delete h;
      return SVGP_ERR_INVALID_ARG;
    }
    for (int k = 0; k < h->gh.n; ++k) {
      h->gh.t[k] = t[k];
      h->gh.w[k] = w[k] / 1.7724538509055160273;   // / sqrt(pi)
    }
  }
  size_t M2 = (size_t)h->Mp * h->Mp;
  size_t Bp = (size_t)(cfg->B_max + 127) / 128 * 128;
  // operand copies: FP32 (SIMT), BF16, or BF16 hi followed by BF16 lo
  size_t lob = M2 * (h->mode == MODE_F32 ? 4 : h->mode == MODE_BF16 ? 2 : 4);
  int W = 2 * cfg->D + 1;
  bool ok = dalloc(h, &h->Kuu_f, M2 * 4) && dalloc(h, &h->Lf, M2 * 4) && dalloc(h, &h->Pf, M2 * 4) &&
            dalloc(h, &h->Psi, M2 * 4) && dalloc(h, &h->GKuu, M2 * 4) && dalloc(h, &h->L_lo, lob) &&
            dalloc(h, &h->Lt_lo, lob) && dalloc(h, &h->V, lob) && dalloc(h, &h->S, lob) &&
            dalloc(h, &h->Y, lob) && dalloc(h, &h->GP_lo, lob) &&
            dalloc(h, &h->Zs, sizeof(float) * h->Mp * h->Dp) && dalloc(h, &h->Xs, sizeof(float) * Bp * h->Dp) &&
            dalloc(h, &h->v, sizeof(float) * h->Mp) && dalloc(h, &h->w, sizeof(float) * h->Mp) &&
            dalloc(h, &h->mu, sizeof(float) * Bp) && dalloc(h, &h->g, sizeof(float) * Bp) &&
            dalloc(h, &h->Kg, sizeof(float) * h->Mp) && dalloc(h, &h->colsum, sizeof(float) * Bp) &&
            dalloc(h, &h->dm_tmp, sizeof(float) * h->Mp) &&
            dalloc(h, &h->rowacc_f, sizeof(float) * h->Mp * W) && dalloc(h, &h->rowacc_u, sizeof(float) * h->Mp * W) &&
            dalloc(h, &h->red, sizeof(double) * RED_COUNT) && dalloc(h, &h->acc_ell, sizeof(double) * SVGP_MAXD) &&
            dalloc(h, &h->resid_tmp, sizeof(double)) && dalloc(h, &h->errword, sizeof(int)) &&
            dalloc(h, &h->done, sizeof(int)) && dalloc(h, &h->iters_tmp, sizeof(int));
  if (ok && h->mode != MODE_F32) ok = dalloc(h, &h->Kuu_lo, h->kuu3 ? lob / 2 * 3 : lob) && dalloc(h, &h->P_lo, lob);
  if (ok) ok = dalloc(h, &h->gapN, M2 * 4);
  if (ok) ok = dalloc(h, &h->hut, sizeof(float) * 3 * (size_t)h->M * SVGP_HUTCH_KMAX);
  h->tc_kuf = h->mode != MODE_F32 && tc_kuf_supported(h->D);
  if (ok && h->tc_kuf)
    ok = dalloc(h, &h->kt.ZR, 2 * 64 * h->Mp) && dalloc(h, &h->kt.ZK, 2 * 64 * h->Mp) &&
         dalloc(h, &h->kt.XR, 2 * 64 * Bp) && dalloc(h, &h->kt.XK, 2 * 64 * Bp) &&
         dalloc(h, &h->rowpart, sizeof(float) * ((size_t)tc_num_sms() * 256 + h->Mp) * W);
  if (ok && h->probit) {
    ok = dalloc(h, &h->hn, sizeof(float) * Bp);
    if (ok && h->tc_kuf) ok = dalloc(h, &h->kt.XKh, 2 * 64 * Bp);
  }
  if (ok && h->mode == MODE_F32) { h->Kuu_lo = h->Kuu_f; h->P_lo = h->Pf; }
  if (ok) ok = build_ctx(h, h->gs, 128, 128, false) && build_ctx(h, h->gt, 128, 128, h->mode != MODE_F32);
  simt_init_attributes();
  if (h->mode != MODE_F32) tc_init_attributes();
  if (h->tc_kuf) tc_kuf_init_attributes();
  if (!ok) {
    svgp_destroy(h);
    return SVGP_ERR_OOM;
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    svgp_destroy(h);
    return SVGP_ERR_CUDA;
  }
  *out = h;
  return SVGP_OK;
}

void svgp_destroy(svgp_handle* h) {
  if (!h) return;
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->st_aux) cudaStreamDestroy(h->st_aux);
  for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
  for (void* p : h->allocs) cudaFree(p);
  delete h;
}

svgp_status svgp_set_stream(svgp_handle* h, void* stream) {
  if (!h) return SVGP_ERR_INVALID_ARG;
  h->st = (cudaStream_t)stream;
  h->gs.st = h->st;
  h->gt.st = h->st;
  return SVGP_OK;
}

int svgp_param_count(const svgp_handle* h) {
  return h ? h->M * h->D + h->D + 2 + 2 * h->M : 0;
}

long long svgp_launch_count(const svgp_handle* h) {
  (void)h;
  return (long long)__atomic_load_n(&g_launches, __ATOMIC_RELAXED);
}

svgp_status svgp_profile_enable(svgp_handle* h, int enable) {
  if (!h) return SVGP_ERR_INVALID_ARG;
  if (enable && h->ev.empty()) {
    h->ev.resize(1024);
    for (auto& e : h->ev)
      if (cudaEventCreate(&e) != cudaSuccess) return fail(h, SVGP_ERR_CUDA, "cudaEventCreate failed");
  }
  h->prof = enable != 0;
  if (enable) h->rec_kind.clear();
  return SVGP_OK;
}

svgp_status svgp_profile_read(svgp_handle* h, float* ms, int* counts) {
  if (!h || !ms || !counts) return SVGP_ERR_INVALID_ARG;
  for (int k = 0; k < SVGP_PROF_NKINDS; ++k) { ms[k] = 0.f; counts[k] = 0; }
  for (size_t r = 0; r < h->rec_kind.size(); ++r) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, h->ev[2 * r], h->ev[2 * r + 1]) != cudaSuccess)
      return fail(h, SVGP_ERR_CUDA, "cudaEventElapsedTime failed (work not complete?)");
    ms[h->rec_kind[r]] += t;
    counts[h->rec_kind[r]] += 1;
  }
  return SVGP_OK;
}

const char* svgp_last_error(const svgp_handle* h) { return h ? h->err : "null handle"; }

svgp_status svgp_bound(svgp_handle* h, const svgp_params* p, const svgp_batch* b, double* terms_dev) {
  if (!h) return SVGP_ERR_INVALID_ARG;
  if (!valid_params(h, p)) return fail(h, SVGP_ERR_INVALID_ARG, "params: null pointer");
  if (!terms_dev) return fail(h, SVGP_ERR_INVALID_ARG, "terms_dev is null");
  svgp_status s = validate_batch(h, b);
  if (s != SVGP_OK) return s;
  prologue(h, p, b->X, b->B, p->L);
  forward(h, p, b, true);
  k_terms_finalize(h->red, h->acc_ell, p->sf2, p->noise, p->ell, h->M, h->D, b->B, b->N, h->probit, 0, terms_dev,
                   nullptr, nullptr, nullptr, h->errword, h->st);
  return check_launch(h, "svgp_bound");
}

svgp_status svgp_bound_hutchinson(svgp_handle* h, const svgp_params* p, const svgp_batch* b, const float* probes,
                                  int K, double* terms_dev) {
  if (!h) return SVGP_ERR_INVALID_ARG;
  if (!valid_params(h, p) || !probes || !terms_dev)
    return fail(h, SVGP_ERR_INVALID_ARG, "bound_hutchinson: null pointer");
  if (K < 1 || K > SVGP_HUTCH_KMAX) return fail(h, SVGP_ERR_INVALID_ARG, "bound_hutchinson: K out of [1, 256]");
  svgp_status s = validate_batch(h, b);
  if (s != SVGP_OK) return s;
  prologue(h, p, b->X, b->B, p->L);
  // no P and no O(M^3) product: the data term from k_n^T P k_n of the
  // factored form per point, the two traces from the probes (Section 3.4)
  cudaStream_t st = h->st;
  const int M = h->M, Mp = h->Mp;
  float* bufA = h->hut;
  float* bufB = h->hut + (size_t)M * SVGP_HUTCH_KMAX;
  float* bufC = h->hut + 2 * (size_t)M * SVGP_HUTCH_KMAX;
  // v = P m~ from vector products (O(M^2)); the B and K column blocks on
  // the tensor cores in the handle's operand precision, else FP32 SIMT
  // (the probe block must fit the transposed M x M buffers: K <= Mp)
  const bool tc = h->mode != MODE_F32 && (K + 127) / 128 * 128 <= Mp;
  k_hutch_data(h->Lf, h->Kuu_f, p->s, M, Mp, h->Zs, h->Xs, h->D, tc ? 0 : b->B, p->sf2, p->m, !h->unprec, bufA,
               bufB, bufC, SVGP_HUTCH_KMAX, h->v, h->colsum, h->red, st);
  if (tc) {
    const bool ok = h->mode == MODE_BF16
                        ? hutch_tc<bf16*>(h, p, b, probes, K, [](void* q) { return H(q); })
                        : hutch_tc<SplitPtr>(h, p, b, probes, K, [h](void* q) { return SP(h, q); });
    if (!ok) return fail(h, SVGP_ERR_CUDA, "bound_hutchinson: tall-skinny schedule or launch failed");
  }
  k_gemv(h->Kuu_f, Mp, M, h->v, 1.f, nullptr, 0.f, h->w, h->v, h->red + RED_QUAD, st);     // w = Kuu v, v^T w
  if (!(h->tc_kuf && tc_kuf_gemv(h->kt.XR, b->B, h->kt.ZK, M, h->v, h->mu, true, h->errword, st)))
    k_mu(h->Zs, h->Xs, M, b->B, h->D, p->sf2, h->v, h->mu, st);                          // mu = Kfu v
  if (h->probit) k_pointwise_probit(b->y, h->mu, h->colsum, p->sf2, b->B, h->gh, h->g, h->hn, h->red, st);
  else k_pointwise_gauss(b->y, h->mu, p->noise, b->B, h->g, h->red, st);
  if (!tc) k_hutchinson(h->Lf, h->Kuu_f, p->s, M, Mp, probes, K, bufA, bufB, bufC, h->red, st);
  k_terms_finalize(h->red, h->acc_ell, p->sf2, p->noise, p->ell, h->M, h->D, b->B, b->N, h->probit, K, terms_dev,
                   nullptr, nullptr, nullptr, h->errword, h->st);
  return check_launch(h, "svgp_bound_hutchinson");
}

svgp_status svgp_backward(svgp_handle* h, const svgp_params* p, const svgp_batch* b, double* terms_dev,
                          const svgp_grads* gr) {
  if (!h) return SVGP_ERR_INVALID_ARG;
  if (!valid_params(h, p)) return fail(h, SVGP_ERR_INVALID_ARG, "params: null pointer");
  if (!valid_grads(gr)) return fail(h, SVGP_ERR_INVALID_ARG, "grads: null pointer");
  svgp_status s = validate_batch(h, b);
  if (s != SVGP_OK) return s;
  prologue(h, p, b->X, b->B, p->L);
  backward_tail(h, p, b, terms_dev, gr);
  return check_launch(h, "svgp_backward");
}

svgp_status svgp_ng_update_T(svgp_handle* h, const svgp_params* p, float* L_inout, const float* gamma_dev,
                             int max_iters, double eps, int* iters_dev, double* residual_dev) {
  if (!h) return SVGP_ERR_INVALID_ARG;
  if (!valid_ng_args(p, L_inout, gamma_dev, max_iters))
    return fail(h, SVGP_ERR_INVALID_ARG, "ng_update_T: null pointer or max_iters out of [0, 100000]");
  prologue(h, p, nullptr, 0, L_inout);
  ng_loop(h, p, L_inout, gamma_dev, max_iters, eps, iters_dev ? iters_dev : h->iters_tmp,
          residual_dev ? residual_dev : h->resid_tmp);
  return check_launch(h, "svgp_ng_update_T");
}

svgp_status svgp_variance_gap(svgp_handle* h, const svgp_params* p, const svgp_batch* b, double sigma2,
                              double* gap_dev) {
  if (!h) return SVGP_ERR_INVALID_ARG;
  if (!valid_params(h, p) || !gap_dev) return fail(h, SVGP_ERR_INVALID_ARG, "variance_gap: null pointer");
  svgp_status s = validate_batch(h, b);
  if (s != SVGP_OK) return s;
  cudaStream_t st = h->st;
  prologue(h, p, b->X, b->B, p->L);
  run_psi(h, p, b->B, nullptr);
  k_kt_f32(h->Kuu_f, p->s, h->M, h->Mp, h->GKuu, st);
  gap_compute(h, nullptr);   // red[RED_GAPDOT] is 0 after the prologue
  k_gap_check(h->red, p->s, h->M, sigma2, p->noise, 0.0, nullptr, gap_dev, st);
  return check_launch(h, "svgp_variance_gap");
}

svgp_status svgp_ng_update_T_gap(svgp_handle* h, const svgp_params* p, const svgp_batch* b, float* L_inout,
                                 const float* gamma_dev, int max_iters, double eps, double sigma2, int* iters_dev,
                                 double* gap_dev) {
  if (!h) return SVGP_ERR_INVALID_ARG;
  if (!valid_ng_args(p, L_inout, gamma_dev, max_iters) || !p->noise)
    return fail(h, SVGP_ERR_INVALID_ARG, "ng_update_T_gap: null pointer or max_iters out of [0, 100000]");
  if (h->probit) return fail(h, SVGP_ERR_UNSUPPORTED, "ng_update_T_gap: the gap rule is for the Gaussian likelihood");
  svgp_status s = validate_batch(h, b);
  if (s != SVGP_OK) return s;
  cudaStream_t st = h->st;
  int* iters = iters_dev ? iters_dev : h->iters_tmp;
  prologue(h, p, b->X, b->B, L_inout);
  run_psi(h, p, b->B, nullptr);
  k_kt_f32(h->Kuu_f, p->s, h->M, h->Mp, h->GKuu, st);
  k_zero(st, h->done, sizeof(int), iters, sizeof(int));
  for (int t = 0; t <= max_iters; ++t) {
    // G(L_t); stop before updating once G <= 2 noise eps (the last pass only measures)
    if (t > 0) k_zero(st, h->red + RED_GAPDOT, sizeof(double));
    gap_compute(h, h->done);
    k_gap_check(h->red, p->s, h->M, sigma2, p->noise, eps, h->done, gap_dev, st);
    if (t == max_iters) break;
    run_vt(h, h->Kuu_lo, p->s, h->done);
    run_sym<0>(h, h->done);
    k_ng_check(h->red, h->M, 0.0, h->done, iters, h->resid_tmp, h->errword, st);
    run_lupd(h, L_inout, gamma_dev + t);
    prep_L(h, L_inout, nullptr);
  }
  return check_launch(h, "svgp_ng_update_T_gap");
}

svgp_status svgp_train_step(svgp_handle* h, const svgp_params* p, const svgp_batch* b, float* L_inout,
                            const float* gamma_dev, int max_iters, double eps, int* iters_dev, double* residual_dev,
                            double* terms_dev, const svgp_grads* gr) {
  if (!h) return SVGP_ERR_INVALID_ARG;
  if (!valid_params(h, p) || !valid_ng_args(p, L_inout, gamma_dev, max_iters))
    return fail(h, SVGP_ERR_INVALID_ARG, "train_step: null pointer or max_iters out of [0, 100000]");
  if (!valid_grads(gr)) return fail(h, SVGP_ERR_INVALID_ARG, "grads: null pointer");
  svgp_status s = validate_batch(h, b);
  if (s != SVGP_OK) return s;
  // one prologue (coordinates, Kuu, Kuf generator operands, L copies) serves both parts
  // the log-det of L is taken after the NG update (the prologue's is of the old L)
  int* iters = iters_dev ? iters_dev : h->iters_tmp;
  prologue(h, p, b->X, b->B, L_inout, max_iters == 0, h->done, iters);
  fork_psi(h, p, b->B);   // overlaps the NG update; joined before P in the forward pass
  ng_loop(h, p, L_inout, gamma_dev, max_iters, eps, iters, residual_dev ? residual_dev : h->resid_tmp, true);
  if (max_iters > 0) prep_L(h, L_inout, h->red + RED_LOGDETL);   // copies and log-det of the updated L
  svgp_params q = *p;
  q.L = L_inout;
  backward_tail(h, &q, b, terms_dev, gr);
  return check_launch(h, "svgp_train_step");
}

svgp_status svgp_predict(svgp_handle* h, const svgp_params* p, const float* Xs, int Ns, float* mean, float* var,
                         int include_noise) {
  if (!h) return SVGP_ERR_INVALID_ARG;
  if (!valid_params(h, p) || !Xs || !mean || !var) return fail(h, SVGP_ERR_INVALID_ARG, "predict: null pointer");
  if (Ns < 1 || Ns > h->Bmax) return fail(h, SVGP_ERR_INVALID_ARG, "predict: Ns out of [1, B_max]");
  cudaStream_t st = h->st;
  prologue(h, p, Xs, Ns, p->L);
  forward(h, p, nullptr, false);
  if (!(h->tc_kuf && tc_kuf_gemv(h->kt.XR, Ns, h->kt.ZK, h->M, h->v, mean, false, h->errword, st)))
    k_mu(h->Zs, h->Xs, h->M, Ns, h->D, p->sf2, h->v, mean, st);
  k_zero(st, h->colsum, sizeof(float) * Ns);
  WEpi we{KufGen{h->Zs, h->Xs, h->D, h->M, Ns, p->sf2}, nullptr, nullptr, nullptr, nullptr, 0.f,
          nullptr, h->colsum};
  run_w(h, we);
  k_predict_finalize(h->colsum, p->sf2, p->noise, Ns, include_noise, var, st);
  return check_launch(h, "svgp_predict");
}

svgp_status svgp_adam_step(svgp_handle* h, float* raw, float* constrained, const float* grad, float* m1, float* m2,
                           int* step_dev, const float* hyper_dev, const float* zbeta1_dev) {
  if (!h) return SVGP_ERR_INVALID_ARG;
  if (!raw || !constrained || !grad || !m1 || !m2 || !step_dev || !hyper_dev)
    return fail(h, SVGP_ERR_INVALID_ARG, "adam: null pointer");
  k_adam(raw, constrained, grad, m1, m2, step_dev, hyper_dev, zbeta1_dev, h->M, h->D, h->st);
  return check_launch(h, "svgp_adam_step");
}

namespace {
// Tile table of a contraction kind (SVGP_PROF_*), or -1.
int kind_table(int kind) {
  switch (kind) {
    case SVGP_PROF_VT: return TT_VT;
    case SVGP_PROF_SYM: return TT_SYM_IN;
    case SVGP_PROF_LUPD: return TT_LUPD;
    case SVGP_PROF_LS: return TT_LS;
    case SVGP_PROF_OUT: return TT_OUT;
    default: return -1;
  }
}
}  // namespace

int svgp_split_candidates(const svgp_handle* h, int kind, int* out, int n) {
  const int t = kind_table(kind);
  if (!h || t < 0 || h->mode == MODE_F32) return 0;
  std::vector<int> c = h->may_split[t] ? split_candidates(h->tc_tiles[t]) : std::vector<int>{0};
  for (int i = 0; i < (int)c.size() && i < n && out; ++i) out[i] = c[i];
  return (int)c.size();
}

int svgp_get_split(const svgp_handle* h, int kind) {
  const int t = kind_table(kind);
  if (!h || t < 0 || h->mode == MODE_F32) return -1;
  return h->tc_kmin[t];
}

svgp_status svgp_set_split(svgp_handle* h, int kind, int kmin) {
  if (!h) return SVGP_ERR_INVALID_ARG;
  const int t = kind_table(kind);
  if (t < 0) return fail(h, SVGP_ERR_INVALID_ARG, "set_split: not a tensor-core contraction kind");
  if (h->mode == MODE_F32) return fail(h, SVGP_ERR_UNSUPPORTED, "set_split: FP32 handles have no split schedule");
  if (kmin < 0) kmin = h->may_split[t] ? model_kmin(h->tc_tiles[t], tc_num_sms()) : 0;
  if (kmin > 0 && !h->may_split[t]) return fail(h, SVGP_ERR_INVALID_ARG, "set_split: this kind keeps whole tiles");
  // the stream must be idle: an in-flight launch may read the tables
  if (cudaStreamSynchronize(h->st) != cudaSuccess || cudaStreamSynchronize(h->st_aux) != cudaSuccess)
    return fail(h, SVGP_ERR_CUDA, "set_split: stream synchronisation failed");
  if (!schedule_table(h, t, kmin)) {
    schedule_table(h, t, h->tc_kmin[t]);
    return fail(h, SVGP_ERR_INVALID_ARG, "set_split: threshold below the smallest candidate");
  }
  return SVGP_OK;
}

svgp_status svgp_check_wait_timeout(svgp_handle* h) {
  if (!h) return SVGP_ERR_INVALID_ARG;
  if (!tc_available()) return fail(h, SVGP_ERR_UNSUPPORTED, "check_wait_timeout: no tensor-core device");
  tc_wait_probe(h->errword, h->st);
  return check_launch(h, "svgp_check_wait_timeout");
}

svgp_status svgp_sync_status(svgp_handle* h) {
  if (!h) return SVGP_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(h->st) != cudaSuccess) return fail(h, SVGP_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
  int e = 0;
  if (cudaMemcpy(&e, h->errword, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return SVGP_ERR_CUDA;
  cudaMemset(h->errword, 0, sizeof(int));
  if (e & ERRBIT_TIMEOUT) {
    // a launch that gave up may have left split-K counts behind: clear them
    if (h->gt.kflag) cudaMemset(h->gt.kflag, 0, sizeof(int) * 2 * (size_t)h->gt.nslot);
    return fail(h, SVGP_ERR_TIMEOUT, "a device pipeline wait timed out");
  }
  if (e & ERRBIT_NONFINITE) return fail(h, SVGP_ERR_NONFINITE, "non-finite bound");
  return SVGP_OK;
}

}  // extern "C"
