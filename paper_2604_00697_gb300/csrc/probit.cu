// Bernoulli likelihood with probit link: p(y | f) = Phi(s f), s = 2y - 1 (the
// binary classification experiments of Section 4.1; GPflow's Bernoulli
// likelihood, Appendix S5.3).  Its expectation under q(f_n) = N(mu_n,
// sigma_n^2) of Eq. (7) has no closed form and is taken with a Gauss-Hermite
// rule:
//   E_n = sum_k w_k / sqrt(pi) log Phi(s_n f_nk),  f_nk = mu_n + sqrt(2) sigma_n t_k,
// together with the derivatives the backward pass needs (the derivatives of
// the rule itself, so that they are exact for the computed bound):
//   g_n = dE_n/dmu_n      = sum_k w_k / sqrt(pi) s_n r(s_n f_nk)
//   h_n = dE_n/dsigma_n^2 = sum_k w_k / sqrt(pi) s_n r(s_n f_nk) t_k / (sqrt(2) sigma_n)
// with r = phi / Phi (the derivative of log Phi).  For sigma_n below 1e-6 the
// last quotient is replaced by its limit 1/2 sum_k w_k / sqrt(pi) r'(s_n f_nk),
// r'(a) = -r(a) (a + r(a)).  Everything per point is FP64.
#include <math.h>

#include <vector>

#include "common.cuh"
#include "internal.h"

// ---------------------------------------------------------------------------
// Gauss-Hermite rule for the weight exp(-t^2) (host).
//
// The orthonormal polynomials q_j for this weight satisfy
//   q_0 = pi^(-1/4),  q_{j+1}(t) = sqrt(2/(j+1)) t q_j(t) - sqrt(j/(j+1)) q_{j-1}(t),
// and q_n' = sqrt(2n) q_{n-1}.  The nodes are the n roots of q_n (all inside
// |t| < sqrt(2n + 1)); each is bracketed by a sign change on a fine grid,
// narrowed by bisection and polished by Newton's method.  The Christoffel
// weights are w_k = 1 / (n q_{n-1}(t_k)^2).
// ---------------------------------------------------------------------------
namespace {

void hermite_q(int n, double t, double* qn, double* qn1) {
  double qm = 0.0, q = 0.7511255444649425;   // pi^(-1/4)
  for (int j = 0; j < n; ++j) {
    const double qp = sqrt(2.0 / (j + 1)) * t * q - sqrt((double)j / (j + 1)) * qm;
    qm = q;
    q = qp;
  }
  *qn = q;
  *qn1 = qm;
}

}  // namespace

bool gauss_hermite_rule(int n, double* t, double* w) {
  if (n < 1 || n > 64 || !t || !w) return false;
  const double lim = sqrt(2.0 * n + 1.0) + 0.5;
  const int steps = 4000 * n;
  const double h = 2.0 * lim / steps;
  // the grid is shifted by a fraction of a step so that no grid point lands
  // on the root at t = 0 of odd n; a zero value counts as non-negative
  int found = 0;
  double a = -lim - 0.37 * h, qa, qa1;
  hermite_q(n, a, &qa, &qa1);
  for (int i = 1; i <= steps + 1 && found < n; ++i) {
    const double b = a + h;
    double qb, qb1;
    hermite_q(n, b, &qb, &qb1);
    if ((qa < 0.0) != (qb < 0.0)) {
      double lo = a, hi = b, flo = qa;
      for (int it = 0; it < 60; ++it) {
        const double mid = 0.5 * (lo + hi);
        double fm, fm1;
        hermite_q(n, mid, &fm, &fm1);
        if ((fm < 0.0) == (flo < 0.0)) { lo = mid; flo = fm; } else { hi = mid; }
      }
      double x = 0.5 * (lo + hi), q, q1;
      for (int it = 0; it < 2; ++it) {
        hermite_q(n, x, &q, &q1);
        const double dq = sqrt(2.0 * n) * q1;
        if (dq != 0.0) x -= q / dq;
      }
      hermite_q(n, x, &q, &q1);
      t[found] = x;
      w[found] = 1.0 / (n * q1 * q1);
      ++found;
    }
    a = b;
    qa = qb;
  }
  return found == n;
}

namespace {

// log Phi(a) and r(a) = phi(a) / Phi(a) in FP64.  Phi(a) = erfc(-a/sqrt 2)/2;
// below a = -1 through the scaled complement erfcx so that neither
// underflows; above 0, log Phi = log1p(-erfc(a/sqrt 2)/2).
__device__ __forceinline__ void log_phi_ratio(double a, double* lp, double* r) {
  const double RSQRT2 = 0.70710678118654752440, SQRT_2_OVER_PI = 0.79788456080286535588,
               RSQRT_2PI = 0.39894228040143267794;
  if (a < -1.0) {
    const double ex = erfcx(-a * RSQRT2);
    *lp = log(0.5 * ex) - 0.5 * a * a;
    *r = SQRT_2_OVER_PI / ex;
  } else {
    const double tail = 0.5 * erfc(a * RSQRT2);          // 1 - Phi(a)
    const double Phi = 1.0 - tail;
    *lp = a > 0.0 ? log1p(-tail) : log(Phi);
    *r = RSQRT_2PI * exp(-0.5 * a * a) / Phi;
  }
}

__global__ void pointwise_probit_kernel(const float* __restrict__ y, const float* __restrict__ mu,
                                        const float* __restrict__ colsum, const float* __restrict__ sf2p, int B,
                                        GHRule gh, float* __restrict__ g, float* __restrict__ h, double* red) {
  pdl_enter();
  const double SQRT2 = 1.41421356237309504880;
  const double sf2 = *sf2p;
  double sE = 0.0, sH = 0.0, sV = 0.0, sC = 0.0;
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < B; n += gridDim.x * blockDim.x) {
    const double s = y[n] > 0.5f ? 1.0 : -1.0;
    double var = sf2 - (double)colsum[n];
    if (var < 0.0) { var = 0.0; sC += 1.0; }
    const double sd = sqrt(var), m = mu[n];
    double E = 0.0, G = 0.0, H = 0.0, H2 = 0.0;
    for (int k = 0; k < gh.n; ++k) {
      const double a = s * (m + SQRT2 * sd * gh.t[k]);
      double lp, r;
      log_phi_ratio(a, &lp, &r);
      E += gh.w[k] * lp;
      G += gh.w[k] * r;
      H += gh.w[k] * r * gh.t[k];
      H2 -= gh.w[k] * r * (a + r);
    }
    const double hn = sd >= 1e-6 ? s * H / (SQRT2 * sd) : 0.5 * H2;
    g[n] = (float)(s * G);
    h[n] = (float)hn;
    sE += E;
    sH += hn;
    sV += var;
  }
  block_add_double(sE, red + RED_ELL);
  block_add_double(sH, red + RED_SUMH);
  block_add_double(sV, red + RED_SUMVAR);
  block_add_double(sC, red + RED_NCLAMP);
}

}  // namespace

void k_pointwise_probit(const float* y, const float* mu, const float* colsum, const float* sf2, int B,
                        const GHRule& gh, float* g, float* h, double* red, cudaStream_t st) {
  int grid = (B + 255) / 256;
  if (grid > 1024) grid = 1024;
  svgp_note_launch();
  pdl_launch(pointwise_probit_kernel, grid, 256, 0, st, y, mu, colsum, sf2, B, gh, g, h, red);
}
