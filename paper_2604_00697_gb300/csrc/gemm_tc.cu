// tcgen05 BF16 GEMMs (placeholder until the tensor-core mainloop lands).
#include "common.cuh"
#include "internal.h"

bool tc_available() { return false; }
void tc_init_attributes() {}
bool tc_vt(const GemmCtx&, const bf16*, const bf16*, EpiVt<bf16>) { return false; }
bool tc_sym_ng(const GemmCtx&, const bf16*, const bf16*, EpiSym<bf16, 0>) { return false; }
bool tc_sym_fwd(const GemmCtx&, const bf16*, const bf16*, EpiSym<bf16, 1>) { return false; }
bool tc_sym_bwd(const GemmCtx&, const bf16*, const bf16*, EpiSym<bf16, 2>) { return false; }
bool tc_lupd(const GemmCtx&, const bf16*, const bf16*, EpiLupd) { return false; }
bool tc_ls(const GemmCtx&, const bf16*, const bf16*, EpiStore<bf16>) { return false; }
bool tc_p(const GemmCtx&, const bf16*, const bf16*, EpiP<bf16>) { return false; }
bool tc_gk(const GemmCtx&, const bf16*, const bf16*, EpiGK) { return false; }
bool tc_psi(const GemmCtx&, const KufGen&, int, EpiPsi) { return false; }
bool tc_w(const GemmCtx&, const bf16*, const WEpi&) { return false; }
