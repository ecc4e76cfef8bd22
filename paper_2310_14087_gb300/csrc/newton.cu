// Pieces of the Newton direction (Algorithm 1): the weights of the operator T_k (Sec. 4.3) in
// the cost-reduced G + G^T form and in the complement form, and the alpha / alpha-bar split.
#include "kot_internal.cuh"

namespace kot {

namespace {

inline int cdiv(size_t a, int b) { return (int)((a + b - 1) / b); }

// xi_ij = eta_ij / (mu + 1 - eta_ij), eta_ij = sig_i / (sig_i - sig_j), i in alpha, j in alpha-bar
__device__ __forceinline__ double xi_of(double si, double sj, double mu) {
  const double eta = si / (si - sj);
  return eta / (mu + 1.0 - eta);
}

// V: rows x l.  G + G^T form (complement = 0): row r is eigen-index nb + r (in alpha); column j in
// alpha (j >= nb) is scaled by 1/(2 mu), column j in alpha-bar by xi(sig_{nb+r}, sig_j).
// Complement form (complement = 1): row r is eigen-index r (in alpha-bar); column j in alpha-bar
// is scaled by 1/(2 mu), column j in alpha by 1/mu - xi(sig_j, sig_r).
__global__ void k_t_weights(int rows, int l, int nb, const double* __restrict__ sig, double mu,
                            int complement, double* __restrict__ V) {
  pdl_wait();
  pdl_trigger();
  const int j = blockIdx.x * 32 + threadIdx.x, r = blockIdx.y * 8 + threadIdx.y;
  if (r >= rows || j >= l) return;
  double w;
  if (!complement) {
    const int i = nb + r;
    w = (j >= nb) ? 0.5 / mu : xi_of(sig[i], sig[j], mu);
  } else {
    const int i = r;
    w = (j < nb) ? 0.5 / mu : (1.0 / mu - xi_of(sig[j], sig[i], mu));
  }
  V[(size_t)r * l + j] *= w;
}

// A2 = -(1 + Psi) o B / (mu + 1) over l x l (Psi of Sec. 4.3: 1/mu on alpha x alpha, xi on
// alpha x alpha-bar and its transpose, 0 on alpha-bar x alpha-bar; eigen-index i < nb is in
// alpha-bar)
__global__ void k_rhs_weights(int l, int nb, const double* __restrict__ sig, double mu,
                              const double* __restrict__ B, double* __restrict__ A2) {
  pdl_wait();
  pdl_trigger();
  const int j = blockIdx.x * 32 + threadIdx.x, i = blockIdx.y * 8 + threadIdx.y;
  if (i >= l || j >= l) return;
  const bool ai = i >= nb, aj = j >= nb;
  double psi = 0.0;
  if (ai && aj) psi = 1.0 / mu;
  else if (ai) psi = xi_of(sig[i], sig[j], mu);
  else if (aj) psi = xi_of(sig[j], sig[i], mu);
  const size_t o = (size_t)i * l + j;
  A2[o] = -(1.0 + psi) * B[o] / (mu + 1.0);
}

// D = A2 - P^T T[Phi*(x)] P, the latter given by its alpha rows Wx (|alpha| x l, the
// alpha x alpha block halved): 2 Wx on alpha x alpha, Wx on alpha x alpha-bar, Wx^T on
// alpha-bar x alpha, 0 on alpha-bar x alpha-bar.
__global__ void k_assemble_dir(int l, int nb, const double* __restrict__ A2, const double* __restrict__ Wx,
                               double* __restrict__ D) {
  pdl_wait();
  pdl_trigger();
  const int j = blockIdx.x * 32 + threadIdx.x, i = blockIdx.y * 8 + threadIdx.y;
  if (i >= l || j >= l) return;
  double w = 0.0;
  if (i >= nb) w = (j >= nb ? 2.0 : 1.0) * Wx[(size_t)(i - nb) * l + j];
  else if (j >= nb) w = Wx[(size_t)(j - nb) * l + i];
  const size_t o = (size_t)i * l + j;
  D[o] = A2[o] - w;
}

__global__ void k_count_nonpos(int l, const double* __restrict__ sig, int* __restrict__ nb) {
  pdl_wait();
  pdl_trigger();
  __shared__ int sh[256];
  int c = 0;
  for (int i = threadIdx.x; i < l; i += 256) c += (sig[i] <= 0.0);
  sh[threadIdx.x] = c;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *nb = sh[0];
}

}  // namespace

void t_weights(cudaStream_t st, int l, int nb, const double* sig, double mu, int complement,
               double* V) {
  const int rows = complement ? nb : l - nb;
  if (rows <= 0) return;
  launch_pdl(k_t_weights, dim3(cdiv(l, 32), cdiv(rows, 8)), dim3(32, 8), 0, st, rows, l, nb, sig, mu,
             complement, V);
  KOT_CHECK_LAUNCH();
}

void rhs_weights(cudaStream_t st, int l, int nb, const double* sig, double mu, const double* B, double* A2) {
  launch_pdl(k_rhs_weights, dim3(cdiv(l, 32), cdiv(l, 8)), dim3(32, 8), 0, st, l, nb, sig, mu, B, A2);
  KOT_CHECK_LAUNCH();
}

void assemble_dir(cudaStream_t st, int l, int nb, const double* A2, const double* Wx, double* D) {
  launch_pdl(k_assemble_dir, dim3(cdiv(l, 32), cdiv(l, 8)), dim3(32, 8), 0, st, l, nb, A2, Wx, D);
  KOT_CHECK_LAUNCH();
}

void count_nonpos(cudaStream_t st, int l, const double* sig, int* nb) {
  launch_pdl(k_count_nonpos, dim3(1), dim3(256), 0, st, l, sig, nb);
  KOT_CHECK_LAUNCH();
}

}  // namespace kot
