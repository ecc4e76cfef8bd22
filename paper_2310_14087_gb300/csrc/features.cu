// Feature assembly (Sec. 3): kernel mean embeddings, the embedding norms q^2, the Gram matrices
// Q and K over the filling points, the cost vector c and z, and the upper Cholesky factor R of
// K + eps I.
//
// All sums are accumulated in FP64 in a fixed order (per-CTA partials summed in index order), so
// repeated calls give identical bits.
#include <algorithm>

#include "kot_internal.cuh"

namespace kot {

namespace {

inline int cdiv(size_t a, int b) { return (int)((a + b - 1) / b); }

// w_i = (1/n) sum_j exp(-||s_j - p_i||^2 * inv2s2); one CTA per filling point p_i.
__global__ void k_embed(int n, int d, const double* __restrict__ S, const double* __restrict__ P,
                        double inv2s2, double* __restrict__ w) {
  extern __shared__ double sh[];          // d doubles for p_i, then 256 for the reduction
  double* p = sh;
  double* red = sh + d;
  const int i = blockIdx.x, t = threadIdx.x;
  for (int c = t; c < d; c += blockDim.x) p[c] = P[(size_t)i * d + c];
  __syncthreads();
  double acc = 0.0;
  for (int j = t; j < n; j += blockDim.x) {
    const double* s = S + (size_t)j * d;
    double dist = 0.0;
    for (int c = 0; c < d; ++c) {
      double diff = s[c] - p[c];
      dist = fma(diff, diff, dist);
    }
    acc += exp(-dist * inv2s2);
  }
  red[t] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (t < o) red[t] += red[t + o];
    __syncthreads();
  }
  if (t == 0) w[i] = red[0] / (double)n;
}

// Potential and gradient at query point x_q (one CTA per point):
//   u = (1/(2 l2)) sum_a c_a k(a, x),  grad = (1/(2 l2 sigma^2)) sum_a c_a k(a, x) (a - x),
// over the sources a = S_j (c = 1/n) then Sf_i (c = -gamma_i).  Sources are taken 256 at a
// time: each thread forms one weight c_a k(a, x) in shared memory, then thread c < d adds up
// coordinate c of the tile's weighted sources (coalesced rows); all sums in a fixed order.
__global__ void k_potential(int m, int d, int n, const double* __restrict__ S, int l,
                            const double* __restrict__ Sf, const double* __restrict__ gamma,
                            const double* __restrict__ Pq, double inv2s2, double scale_u,
                            double scale_g, double* __restrict__ u, double* __restrict__ grad,
                            double* __restrict__ tmap) {
  extern __shared__ double sh[];          // x (d), weights (256), reduction (256), coordinate sums (d)
  double* x = sh;
  double* wt = sh + d;
  double* red = wt + 256;
  double* g1 = red + 256;
  const int q = blockIdx.x, t = threadIdx.x;
  for (int c = t; c < d; c += 256) {
    x[c] = Pq[(size_t)q * d + c];
    g1[c] = 0.0;
  }
  __syncthreads();
  double s0 = 0.0;
  const int total = n + l;
  for (int a0 = 0; a0 < total; a0 += 256) {
    const int a = a0 + t;
    double w = 0.0;
    if (a < total) {
      const double* src = a < n ? S + (size_t)a * d : Sf + (size_t)(a - n) * d;
      double dist = 0.0;
      for (int c = 0; c < d; ++c) {
        const double diff = src[c] - x[c];
        dist = fma(diff, diff, dist);
      }
      w = (a < n ? 1.0 / (double)n : -gamma[a - n]) * exp(-dist * inv2s2);
    }
    wt[t] = w;
    s0 += w;
    __syncthreads();
    if (grad || tmap) {
      const int cnt = min(256, total - a0);
      for (int c = t; c < d; c += 256) {
        double acc = g1[c];
        for (int b = 0; b < cnt; ++b) {
          const int ab = a0 + b;
          const double* src = ab < n ? S + (size_t)ab * d : Sf + (size_t)(ab - n) * d;
          acc = fma(wt[b], src[c], acc);
        }
        g1[c] = acc;
      }
    }
    __syncthreads();
  }
  red[t] = s0;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (t < o) red[t] += red[t + o];
    __syncthreads();
  }
  const double S0 = red[0];
  if (t == 0 && u) u[q] = scale_u * S0;
  for (int c = t; c < d; c += 256) {
    const double gc = scale_g * (g1[c] - S0 * x[c]);
    if (grad) grad[(size_t)q * d + c] = gc;
    if (tmap) tmap[(size_t)q * d + c] = x[c] - gc;
  }
}

// Pair sums over 64 x 64 tiles (I, J) of the n x n kernel matrix, J >= I; off-diagonal tiles
// count twice.  partial[I * nb + J] receives the tile's weighted sum (zero for J < I).
constexpr int PT = 64;
__global__ void k_pair_tiles(int n, int d, const double* __restrict__ S, double inv2s2,
                             double* __restrict__ partial) {
  __shared__ double red[256];
  const int nb = gridDim.x, I = blockIdx.y, J = blockIdx.x, t = threadIdx.x;
  double acc = 0.0;
  if (J >= I) {
    for (int e = t; e < PT * PT; e += 256) {
      int i = I * PT + e / PT, j = J * PT + e % PT;
      if (i < n && j < n) {
        const double* a = S + (size_t)i * d;
        const double* b = S + (size_t)j * d;
        double dist = 0.0;
        for (int c = 0; c < d; ++c) {
          double diff = a[c] - b[c];
          dist = fma(diff, diff, dist);
        }
        acc += exp(-dist * inv2s2);
      }
    }
    if (J > I) acc *= 2.0;
  }
  red[t] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (t < o) red[t] += red[t + o];
    __syncthreads();
  }
  if (t == 0) partial[(size_t)I * nb + J] = red[0];
}

__global__ void k_sum_scaled(int m, const double* __restrict__ partial, double scale,
                             double* __restrict__ out) {
  __shared__ double red[256];
  const int t = threadIdx.x;
  double acc = 0.0;
  for (int i = t; i < m; i += 256) acc += partial[i];
  red[t] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (t < o) red[t] += red[t + o];
    __syncthreads();
  }
  if (t == 0) *out = red[0] * scale;
}

// Q_ij = k(xf_i, xf_j) + k(yf_i, yf_j), K_ij = k((xf_i, yf_i), (xf_j, yf_j)).  Both are symmetric
// and (a - b)^2 = (b - a)^2 exactly, so each pair i <= j is evaluated once and stored at both
// positions (half the FP64 work of the full square, which bounds this kernel); blocks wholly below
// the diagonal exit at once.
__global__ void k_gram(int l, int d, const double* __restrict__ Xf, const double* __restrict__ Yf,
                       double inv2s2, double* __restrict__ Q, double* __restrict__ K) {
  const int j = blockIdx.x * 32 + threadIdx.x, i = blockIdx.y * 8 + threadIdx.y;
  if (i >= l || j >= l || j < i) return;
  double dx = 0.0, dy = 0.0;
  for (int c = 0; c < d; ++c) {
    double a = Xf[(size_t)i * d + c] - Xf[(size_t)j * d + c];
    dx = fma(a, a, dx);
  }
  for (int c = 0; c < d; ++c) {
    double b = Yf[(size_t)i * d + c] - Yf[(size_t)j * d + c];
    dy = fma(b, b, dy);
  }
  const double q = exp(-dx * inv2s2) + exp(-dy * inv2s2), k = exp(-(dx + dy) * inv2s2);
  Q[(size_t)i * l + j] = q;
  K[(size_t)i * l + j] = k;
  if (j != i) {
    Q[(size_t)j * l + i] = q;
    K[(size_t)j * l + i] = k;
  }
}

// The same Gram matrices with the distances and exponentials in FP32 (the stored values are the
// FP32 results, exactly, in FP64): FP32 issues about 32x the FP64 rate here, so this build is
// bound by its stores instead of the FP64 pipe.  A block covers a 64 x 64 tile of pairs with 256
// threads, each a 4 x 4 register tile; the tile's 64 + 64 points are staged in shared memory as
// FP32, GW coordinates at a time.  Only tiles that reach the diagonal or above run, and each pair
// i <= j is stored at both positions.
constexpr int GT = 64, GW = 32;
__global__ void __launch_bounds__(256) k_gram_f32(int l, int d, const double* __restrict__ Xf,
                                                  const double* __restrict__ Yf, float inv2s2,
                                                  double* __restrict__ Q, double* __restrict__ K) {
  const int bi = blockIdx.y * GT, bj = blockIdx.x * GT;
  if (bj + GT <= bi) return;                       // wholly below the diagonal
  __shared__ float pr[2][GW][GT + 1], pc[2][GW][GT + 1];   // [x or y][coordinate][point]
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;   // 16 x 16 threads, 4 x 4 pairs each
  float dx[4][4] = {}, dy[4][4] = {};
  for (int c0 = 0; c0 < d; c0 += GW) {
    __syncthreads();
    for (int e = threadIdx.x; e < 2 * GW * GT; e += 256) {
      const int h = e / (GW * GT), r = e % (GW * GT), pt = r / GW, c = r % GW;
      const double* S = h ? Yf : Xf;
      const int gi = bi + pt, gj = bj + pt, cc = c0 + c;
      pr[h][c][pt] = (gi < l && cc < d) ? (float)S[(size_t)gi * d + cc] : 0.0f;
      pc[h][c][pt] = (gj < l && cc < d) ? (float)S[(size_t)gj * d + cc] : 0.0f;
    }
    __syncthreads();
    const int cn = min(GW, d - c0);
    for (int c = 0; c < cn; ++c) {
      float ax[4], ay[4], bx[4], by[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        ax[u] = pr[0][c][ty * 4 + u];
        ay[u] = pr[1][c][ty * 4 + u];
        bx[u] = pc[0][c][tx * 4 + u];
        by[u] = pc[1][c][tx * 4 + u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const float ex = ax[u] - bx[v], ey = ay[u] - by[v];
          dx[u][v] = fmaf(ex, ex, dx[u][v]);
          dy[u][v] = fmaf(ey, ey, dy[u][v]);
        }
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = bi + ty * 4 + u;
    if (i >= l) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int j = bj + tx * 4 + v;
      if (j >= l || j < i) continue;
      const double q = (double)(expf(-dx[u][v] * inv2s2) + expf(-dy[u][v] * inv2s2));
      const double k = (double)expf(-(dx[u][v] + dy[u][v]) * inv2s2);
      Q[(size_t)i * l + j] = q;
      K[(size_t)i * l + j] = k;
      if (j != i) {
        Q[(size_t)j * l + i] = q;
        K[(size_t)j * l + i] = k;
      }
    }
  }
}

// c_i = ||xf_i - yf_i||^2 ; z_i = w_mu_i + w_nu_i - lambda2 c_i
__global__ void k_cost_z(int l, int d, const double* __restrict__ Xf, const double* __restrict__ Yf,
                         double lambda2, const double* __restrict__ w_mu,
                         const double* __restrict__ w_nu, double* __restrict__ c,
                         double* __restrict__ z) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= l) return;
  double s = 0.0;
  for (int k = 0; k < d; ++k) {
    double a = Xf[(size_t)i * d + k] - Yf[(size_t)i * d + k];
    s = fma(a, a, s);
  }
  c[i] = s;
  z[i] = w_mu[i] + w_nu[i] - lambda2 * s;
}

// ------------------------------------------------------------------ blocked upper Cholesky
constexpr int CB = 32;

// Factor the diagonal block A[k0:k0+nb, k0:k0+nb] (upper) in shared memory.  Each pivot's square
// root and reciprocal are formed once, by one thread, and the row is scaled by multiplication: this
// SM issues about two FP64 operations per clock, so a square root or division in every thread
// would cost thousands of cycles per pivot.
__global__ void k_chol_diag(int l, int k0, double* __restrict__ A, int* __restrict__ info) {
  __shared__ double a[CB][CB + 1];
  __shared__ double rinv[2];   // [sqrt(pivot), 1/sqrt(pivot)]
  const int nb = min(CB, l - k0);
  const int tx = threadIdx.x, ty = threadIdx.y;      // 32 x 32
  if (tx < nb && ty < nb) a[ty][tx] = A[(size_t)(k0 + ty) * l + k0 + tx];
  __syncthreads();
  for (int p = 0; p < nb; ++p) {
    if (tx == 0 && ty == 0) {
      double piv = a[p][p];
      if (!(piv > 0.0) || !isfinite(piv)) {
        if (*info == 0) *info = k0 + p + 1;
        piv = 1.0;                                       // keep going; result is discarded
      }
      const double r = sqrt(piv);
      rinv[0] = r;
      rinv[1] = 1.0 / r;
    }
    __syncthreads();
    if (ty == 0 && tx >= p && tx < nb) a[p][tx] = (tx == p) ? rinv[0] : a[p][tx] * rinv[1];
    __syncthreads();
    if (ty > p && tx >= ty && tx < nb && ty < nb) a[ty][tx] -= a[p][ty] * a[p][tx];
    __syncthreads();
  }
  if (tx < nb && ty < nb) A[(size_t)(k0 + ty) * l + k0 + tx] = (tx >= ty) ? a[ty][tx] : 0.0;
}

// Panel: solve R_kk^T X = A[k0:k0+nb, c] for every column c >= k0 + nb (forward substitution).
__global__ void k_chol_panel(int l, int k0, double* __restrict__ A) {
  const int nb = min(CB, l - k0);
  const int col = k0 + nb + blockIdx.x * blockDim.x + threadIdx.x;
  __shared__ double r[CB][CB + 1];
  __shared__ double dinv[CB];   // reciprocals of the diagonal (one division per pivot, not per column)
  for (int e = threadIdx.x; e < CB * CB; e += blockDim.x) {
    int i = e / CB, j = e % CB;
    r[i][j] = (i < nb && j < nb) ? A[(size_t)(k0 + i) * l + k0 + j] : 0.0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < CB; i += blockDim.x) dinv[i] = i < nb ? 1.0 / r[i][i] : 0.0;
  __syncthreads();
  if (col >= l) return;
  double x[CB];
#pragma unroll
  for (int i = 0; i < CB; ++i) {
    if (i < nb) {
      double v = A[(size_t)(k0 + i) * l + col];
      for (int k = 0; k < i; ++k) v -= r[k][i] * x[k];
      x[i] = v * dinv[i];
      A[(size_t)(k0 + i) * l + col] = x[i];
    }
  }
}

__global__ void k_zero_lower(int l, double* A) {
  const int j = blockIdx.x * 32 + threadIdx.x, i = blockIdx.y * 8 + threadIdx.y;
  if (i < l && j < l && j < i) A[(size_t)i * l + j] = 0.0;
}

__global__ void k_rowsums(int l, const double* __restrict__ Q, const double* __restrict__ Kt,
                          double* __restrict__ rs) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= l) return;
  double a = 0.0, b = 0.0;
  for (int j = lane; j < l; j += 32) {
    a += fabs(Q[(size_t)warp * l + j]);
    double k = Kt[(size_t)warp * l + j];
    b = fma(k, k, b);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  if (lane == 0) {
    rs[warp] = a;
    rs[l + warp] = b;
  }
}

__global__ void k_rowmax(int l, const double* __restrict__ rs, double* __restrict__ out2) {
  __shared__ double m1[256], m2[256];
  const int t = threadIdx.x;
  double a = 0.0, b = 0.0;
  for (int i = t; i < l; i += 256) {
    a = fmax(a, rs[i]);
    b = fmax(b, rs[l + i]);
  }
  m1[t] = a;
  m2[t] = b;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (t < o) {
      m1[t] = fmax(m1[t], m1[t + o]);
      m2[t] = fmax(m2[t], m2[t + o]);
    }
    __syncthreads();
  }
  if (t == 0) {
    out2[0] = m1[0];
    out2[1] = m2[0];
  }
}

}  // namespace

void embed_f64(cudaStream_t st, int n, int d, int l, const double* S, const double* P,
               double inv2s2, double* w) {
  size_t smem = (size_t)(d + 256) * sizeof(double);
  if (smem > 48 * 1024) KOT_CUDA(cudaFuncSetAttribute(k_embed, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  ProfScope ps(st, KC_EMBED, (double)n * l * (3.0 * d + 2.0), 8.0 * ((double)n * d + (double)l * d + l));
  k_embed<<<l, 256, smem, st>>>(n, d, S, P, inv2s2, w);
  KOT_CHECK_LAUNCH();
}

void potential_f64(cudaStream_t st, int m, int d, int n, const double* S, int l, const double* Sf,
                   const double* gamma, const double* Pq, double sigma, double lambda2, double* u,
                   double* grad, double* tmap) {
  if (m <= 0) return;
  const size_t smem = (size_t)(2 * d + 512) * sizeof(double);
  if (smem > 48 * 1024)
    KOT_CUDA(cudaFuncSetAttribute(k_potential, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const double inv2s2 = 1.0 / (2.0 * sigma * sigma);
  const double scale_u = 1.0 / (2.0 * lambda2), scale_g = 1.0 / (2.0 * lambda2 * sigma * sigma);
  ProfScope ps(st, KC_EMBED, (double)m * (n + l) * (5.0 * d + 4.0), 8.0 * ((double)(n + l + 2 * m) * d + l));
  k_potential<<<m, 256, smem, st>>>(m, d, n, S, l, Sf, gamma, Pq, inv2s2, scale_u, scale_g, u, grad, tmap);
  KOT_CHECK_LAUNCH();
}

int pair_blocks(int n) {
  int nb = cdiv(n, PT);
  return nb * nb;
}

void pair_mean_f64(cudaStream_t st, int n, int d, const double* S, double inv2s2, double* out,
                   double* partial, int partial_cap) {
  const int nb = cdiv(n, PT);
  if (nb * nb > partial_cap) throw Error{KOT_ERR_INVALID, "pair_mean: partial buffer too small"};
  {
    ProfScope ps(st, KC_PAIRS, (double)n * (n + 1) / 2.0 * (3.0 * d + 2.0), 8.0 * (double)n * d);
    k_pair_tiles<<<dim3(nb, nb), 256, 0, st>>>(n, d, S, inv2s2, partial);
  }
  k_sum_scaled<<<1, 256, 0, st>>>(nb * nb, partial, 1.0 / ((double)n * (double)n), out);
  KOT_LAUNCHED(2);
}

void gram_f64(cudaStream_t st, int l, int d, const double* Xf, const double* Yf, double inv2s2,
              double lambda2, const double* w_mu, const double* w_nu, double* Q, double* K,
              double* c, double* z, bool fp32) {
  {
    // flops: the pairs i <= j, 6d + 5 each; bytes: the points in, Q and K out
    ProfScope ps(st, KC_GRAM, (double)l * (l + 1) / 2.0 * (6.0 * d + 5.0), 8.0 * (2.0 * l * d + 2.0 * (double)l * l));
    if (fp32)
      k_gram_f32<<<dim3(cdiv(l, GT), cdiv(l, GT)), 256, 0, st>>>(l, d, Xf, Yf, (float)inv2s2, Q, K);
    else
      k_gram<<<dim3(cdiv(l, 32), cdiv(l, 8)), dim3(32, 8), 0, st>>>(l, d, Xf, Yf, inv2s2, Q, K);
  }
  k_cost_z<<<cdiv(l, 128), 128, 0, st>>>(l, d, Xf, Yf, lambda2, w_mu, w_nu, c, z);
  KOT_LAUNCHED(2);
}

void cost_z_f64(cudaStream_t st, int l, int d, const double* Xf, const double* Yf, double lambda2,
                const double* w_mu, const double* w_nu, double* c, double* z) {
  k_cost_z<<<cdiv(l, 128), 128, 0, st>>>(l, d, Xf, Yf, lambda2, w_mu, w_nu, c, z);
  KOT_CHECK_LAUNCH();
}

void cholesky_upper_f64(cudaStream_t st, int l, double* A, double eps, int* info) {
  KOT_CUDA(cudaMemsetAsync(info, 0, sizeof(int), st));
  add_diag(st, l, eps, A, l);
  for (int k0 = 0; k0 < l; k0 += CB) {
    const int nb = std::min(CB, l - k0);
    {
      ProfScope ps(st, KC_CHOL, nb * (double)nb * nb / 3.0, 16.0 * nb * nb);
      k_chol_diag<<<1, dim3(32, 32), 0, st>>>(l, k0, A, info);
    }
    KOT_CHECK_LAUNCH();
    const int rest = l - k0 - nb;
    if (rest <= 0) break;
    k_chol_panel<<<cdiv(rest, 32), 32, 0, st>>>(l, k0, A);   // one warp per block: more SMs
    KOT_CHECK_LAUNCH();
    // trailing update of the upper triangle: A[k1:, k1:] -= P^T P, P = A[k0:k1, k1:]
    double* Pp = A + (size_t)k0 * l + k0 + nb;
    double* C = A + (size_t)(k0 + nb) * l + k0 + nb;
    gemm_f64(st, true, false, rest, rest, nb, -1.0, Pp, l, Pp, l, nullptr, 1.0, C, l, G_SYM);
  }
  k_zero_lower<<<dim3(cdiv(l, 32), cdiv(l, 8)), dim3(32, 8), 0, st>>>(l, A);
  KOT_CHECK_LAUNCH();
}

void zero_lower(cudaStream_t st, int l, double* A) {
  k_zero_lower<<<dim3(cdiv(l, 32), cdiv(l, 8)), dim3(32, 8), 0, st>>>(l, A);
  KOT_CHECK_LAUNCH();
}

void rowsum_bounds(cudaStream_t st, int l, const double* Q, const double* Kt, double* out2) {
  // the two row-sum arrays live in out2[2 .. 2 + 2l)
  double* rs = out2 + 2;
  k_rowsums<<<cdiv((size_t)l * 32, 256), 256, 0, st>>>(l, Q, Kt, rs);
  k_rowmax<<<1, 256, 0, st>>>(l, rs, out2);
  KOT_LAUNCHED(2);
}

}  // namespace kot
