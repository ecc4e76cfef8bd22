// Pieces of the Newton direction (Algorithm 1): the weights of the operator T_k (Sec. 4.3) in
// the cost-reduced G + G^T form and in the complement form, and the alpha / alpha-bar split.
#include "kot_internal.cuh"

namespace kot {

namespace {

inline int cdiv(size_t a, int b) { return (int)((a + b - 1) / b); }

__device__ double block_sum256(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

// xi_ij = eta_ij / (mu + 1 - eta_ij), eta_ij = sig_i / (sig_i - sig_j), i in alpha, j in alpha-bar
__device__ __forceinline__ double xi_of(double si, double sj, double mu) {
  const double eta = si / (si - sj);
  return eta / (mu + 1.0 - eta);
}

// Weight of entry (r, j) of the carried rows.  G + G^T form (complement = 0): row r is
// eigen-index nb + r (in alpha); column j in alpha (j >= nb) is weighted 1/(2 mu), column j in
// alpha-bar xi(sig_{nb+r}, sig_j).  Complement form (complement = 1; Psi' = E/mu - Psi): row r is
// eigen-index r (in alpha-bar); column j in alpha-bar is weighted 1/(2 mu), column j in alpha
// 1/mu - xi(sig_j, sig_r).
__device__ __forceinline__ double t_weight(int r, int j, int nb, const double* __restrict__ sig, double mu,
                                           int complement) {
  if (!complement) return (j >= nb) ? 0.5 / mu : xi_of(sig[nb + r], sig[j], mu);
  return (j < nb) ? 0.5 / mu : (1.0 / mu - xi_of(sig[j], sig[r], mu));
}

// V = weights o U over rows x l (V may alias U).
__global__ void k_t_weights(int rows, int l, int nb, const double* __restrict__ sig, double mu,
                            int complement, const double* U, double* V) {
  pdl_wait();
  pdl_trigger();
  const int j = blockIdx.x * 32 + threadIdx.x, r = blockIdx.y * 8 + threadIdx.y;
  if (r >= rows || j >= l) return;
  const size_t o = (size_t)r * l + j;
  V[o] = U[o] * t_weight(r, j, nb, sig, mu, complement);
}

// Norms of the CG stopping test in the eigenbasis, complement form (Sec. 4.3, last paragraph):
// with U the alpha-bar rows of Vx = Cb diag(x) Cb^T and W' = weights o U (complement weights),
//   out[1] = ||A2||^2 + sum_{r < nb, j} (4 A2_rj W'_rj + w'_j W'_rj^2 - (4/mu) W'_rj U_rj)
//            - (2/mu) x . Phi(at2) + x^T (Kt o Kt) x / mu^2,   w'_j = 4 (j < nb), 2 (j >= nb),
// which is ||A2 - Psi o Vx||_F^2 = ||at2 - T[Phi*(x)]||_F^2 for orthogonal P; out[0] = |x|^2.
// *base = ||A2||_F^2.  One block writes out directly; several write partial pairs.
__global__ void k_eig_norms_comp(int l, const double* __restrict__ x, int nb, const double* __restrict__ sig,
                                 double mu, const double* __restrict__ A2, const double* __restrict__ U,
                                 const double* __restrict__ KK, const double* __restrict__ phi_at2,
                                 const double* __restrict__ base, double* __restrict__ out) {
  pdl_wait();
  pdl_trigger();
  __shared__ double sh[256];
  double s1 = 0.0, s2 = 0.0, s3 = 0.0;   // |x|^2; the alpha-bar row terms; x^T KK x - 2 mu x.phi
  const size_t stride = (size_t)gridDim.x * 256;
  const size_t t0 = blockIdx.x * 256 + threadIdx.x;
  for (size_t i = t0; i < (size_t)l; i += stride) {
    s1 = fma(x[i], x[i], s1);
    s3 = fma(-2.0 * mu * x[i], phi_at2[i], s3);
  }
  const size_t nr = (size_t)nb * l;
  for (size_t i = t0; i < nr; i += stride) {
    const int r = (int)(i / l), j = (int)(i - (size_t)r * l);
    const double u = U[i], w = u * t_weight(r, j, nb, sig, mu, 1);
    const double a = A2[i];   // rows r < nb of A2 (ld l) are entries i
    s2 += 4.0 * a * w + (j < nb ? 4.0 : 2.0) * w * w - (4.0 / mu) * w * u;
  }
  const size_t n2 = (size_t)l * l;
  for (size_t i = t0; i < n2; i += stride) {
    const int r = (int)(i / l), j = (int)(i - (size_t)r * l);
    s3 = fma(x[r] * KK[i], x[j], s3);
  }
  s2 += s3 / (mu * mu);
  if (base && blockIdx.x == 0 && threadIdx.x == 0) s2 += *base;
  s1 = block_sum256(s1, sh);
  __syncthreads();
  s2 = block_sum256(s2, sh);
  if (threadIdx.x == 0) {
    out[2 * blockIdx.x] = s1;
    out[2 * blockIdx.x + 1] = s2;
  }
}

// ---- the Schur operator of Algorithm 1 in the eigenbasis for few carried rows (<= 32): two FP64
// kernels in place of two tensor-core products and four small launches.  With rows r0 .. r0 + crow
// of Cb = P^T R (the alpha rows, G + G^T form, or the alpha-bar rows, complement form):
//   k_schur_rows:  U[r][j] = sum_k Cb[r0 + r][k] p_k Cb[j][k],  W = weights o U   (one warp per j)
//   k_schur_cols:  Y[r][i] = sum_j W[r][j] Cb[j][i],  v_i = c sum_r Cb[r0 + r][i] Y[r][i],
//                  Hp_i = alpha (H p)_i + mu p_i + v_i                             (one warp per i)
// (c = 2, H = Q, alpha = 1/(2 lambda2) for G + G^T; c = -2, H = H0 = Q/(2 lambda2) + (Kt o Kt)/mu,
// alpha = 1 for the complement form).  A contraction this small is bound by latency, not by the
// multiply rate: 2 crow l^2 FP64 FMAs spread over every SM take a few microseconds, and FP64 makes
// the CG iterates exact instead of three-slice accurate.
__global__ void __launch_bounds__(256) k_schur_rows(int l, int crow, int r0, const double* __restrict__ Cb,
                                                    const double* __restrict__ p, const double* __restrict__ sig,
                                                    double mu, int nb, int complement, double* __restrict__ carry,
                                                    double* __restrict__ W) {
  pdl_wait();
  pdl_trigger();
  const int j = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;   // 8 warps per column j
  if (j >= l) return;
  const double* b = Cb + (size_t)j * l;
  for (int r = warp; r < crow; r += 8) {
    const double* a = Cb + (size_t)(r0 + r) * l;
    double acc0 = 0.0, acc1 = 0.0;
    int k = lane;
    for (; k + 32 < l; k += 64) {   // two independent chains keep loads in flight
      acc0 = fma(a[k] * p[k], b[k], acc0);
      acc1 = fma(a[k + 32] * p[k + 32], b[k + 32], acc1);
    }
    if (k < l) acc0 = fma(a[k] * p[k], b[k], acc0);
    double acc = acc0 + acc1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      const double w = acc * t_weight(r, j, nb, sig, mu, complement);
      W[(size_t)r * l + j] = w;
      carry[(size_t)r * l + j] = complement ? acc : w;
    }
  }
}

__global__ void __launch_bounds__(256) k_schur_cols(int l, int crow, int r0, const double* __restrict__ CbT,
                                                    const double* __restrict__ W, double c,
                                                    const double* __restrict__ H, double alpha,
                                                    const double* __restrict__ p, double mu,
                                                    double* __restrict__ Hp) {
  pdl_wait();
  pdl_trigger();
  __shared__ double part[8][2];
  const int i = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;   // 8 warps per column i
  if (i >= l) return;
  const double* col = CbT + (size_t)i * l;   // column i of Cb
  // rows of W Cb at column i, each weighted by Cb[r0 + r][i]; warp w takes rows w, w + 8, ...
  double v = 0.0;
  for (int r = warp; r < crow; r += 8) {
    const double* w = W + (size_t)r * l;
    double acc0 = 0.0, acc1 = 0.0;
    int j = lane;
    for (; j + 32 < l; j += 64) {
      acc0 = fma(w[j], col[j], acc0);
      acc1 = fma(w[j + 32], col[j + 32], acc1);
    }
    if (j < l) acc0 = fma(w[j], col[j], acc0);
    double acc = acc0 + acc1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    v = fma(col[r0 + r], acc, v);
  }
  // (H p)_i, the k range split over the 8 warps
  const double* h = H + (size_t)i * l;
  double hp = 0.0;
  for (int k = threadIdx.x; k < l; k += 256) hp = fma(h[k], p[k], hp);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) hp += __shfl_xor_sync(0xffffffffu, hp, o);
  if (lane == 0) {
    part[warp][0] = v;
    part[warp][1] = hp;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sv = 0.0, sh = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      sv += part[q][0];
      sh += part[q][1];
    }
    Hp[i] = fma(mu, p[i], alpha * sh) + c * sv;
  }
}

// B = A^T (l x l)
__global__ void k_transpose(int l, const double* __restrict__ A, double* __restrict__ B) {
  pdl_wait();
  pdl_trigger();
  __shared__ double t[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int y = threadIdx.y; y < 32; y += 8) {
    const int i = by + y, j = bx + threadIdx.x;
    if (i < l && j < l) t[y][threadIdx.x] = A[(size_t)i * l + j];
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += 8) {
    const int i = bx + y, j = by + threadIdx.x;
    if (i < l && j < l) B[(size_t)i * l + j] = t[threadIdx.x][y];
  }
}

// D = A2 - Psi o Vx over l x l (Psi of Sec. 4.3: 1/mu on alpha x alpha, xi on alpha x alpha-bar and
// its transpose, 0 on alpha-bar x alpha-bar): the eigenbasis form of dX = at2 - T[Phi*(x)].
__global__ void k_assemble_psi(int l, int nb, const double* __restrict__ sig, double mu,
                               const double* __restrict__ A2, const double* __restrict__ Vx,
                               double* __restrict__ D) {
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
  D[o] = A2[o] - psi * Vx[o];
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
               double* V, const double* U) {
  const int rows = complement ? nb : l - nb;
  if (rows <= 0) return;
  launch_pdl(k_t_weights, dim3(cdiv(l, 32), cdiv(rows, 8)), dim3(32, 8), 0, st, rows, l, nb, sig, mu,
             complement, U ? U : (const double*)V, V);
  KOT_CHECK_LAUNCH();
}

void eig_norms_comp(cudaStream_t st, int l, const double* x, int nb, const double* sig, double mu,
                    const double* A2, const double* U, const double* KK, const double* phi_at2,
                    const double* base, double* out2, double* partial) {
  const size_t n = (size_t)l * l;
  if (n <= 4096) {
    launch_pdl(k_eig_norms_comp, dim3(1), dim3(256), 0, st, l, x, nb, sig, mu, A2, U, KK, phi_at2, base, out2);
    KOT_CHECK_LAUNCH();
    return;
  }
  const int nbk = kReduceBlocks / 2;   // partial holds kReduceBlocks doubles: nbk pairs
  launch_pdl(k_eig_norms_comp, dim3(nbk), dim3(256), 0, st, l, x, nb, sig, mu, A2, U, KK, phi_at2, base,
             partial);
  sum_pairs(st, nbk, partial, out2);
  KOT_LAUNCHED(1);
}

void schur_rows(cudaStream_t st, int l, int crow, int r0, const double* Cb, const double* p, const double* sig,
                double mu, int nb, int complement, double* carry, double* W) {
  launch_pdl(k_schur_rows, dim3(l), dim3(256), 0, st, l, crow, r0, Cb, p, sig, mu, nb, complement, carry, W);
  KOT_CHECK_LAUNCH();
}

void schur_cols(cudaStream_t st, int l, int crow, int r0, const double* CbT, const double* W, double c,
                const double* H, double alpha, const double* p, double mu, double* Hp) {
  launch_pdl(k_schur_cols, dim3(l), dim3(256), 0, st, l, crow, r0, CbT, W, c, H, alpha, p, mu, Hp);
  KOT_CHECK_LAUNCH();
}

void transpose(cudaStream_t st, int l, const double* A, double* B) {
  launch_pdl(k_transpose, dim3(cdiv(l, 32), cdiv(l, 32)), dim3(32, 8), 0, st, l, A, B);
  KOT_CHECK_LAUNCH();
}

void assemble_psi(cudaStream_t st, int l, int nb, const double* sig, double mu, const double* A2,
                  const double* Vx, double* D) {
  launch_pdl(k_assemble_psi, dim3(cdiv(l, 32), cdiv(l, 8)), dim3(32, 8), 0, st, l, nb, sig, mu, A2, Vx, D);
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
