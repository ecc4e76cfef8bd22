// Symmetric eigen-decomposition by parallel cyclic two-sided Jacobi (textbook method: each
// rotation zeroes one off-diagonal pair, Golub & Van Loan's symmetric Schur 2 x 2 step), with
// round-robin ordering so that every round rotates lp/2 disjoint index pairs at once.
//
// Why Jacobi on this GPU: it needs no sequential scalar chain (no tridiagonal QR sweeps), it is
// exact for clustered and repeated eigenvalues (Z = -lambda1 I at the start of the solve), and it
// takes a warm start: the SSN iteration hands in the eigenbasis of the previous, nearby Z, so
// P^T Z P is already nearly diagonal and one or two sweeps finish the job.
//
// Each round updates every 2 x 2 block {p_a, q_a} x {p_b, q_b} of A in place (one thread per
// block, the blocks are disjoint) and every row of V on the rotated columns.
#include <algorithm>
#include <cmath>

#include "kot_internal.cuh"

namespace kot {

namespace {

inline int cdiv(size_t a, int b) { return (int)((a + b - 1) / b); }

// Round-robin (circle method) pairing of lp indices: round r, slot k.
__device__ __forceinline__ void round_pair(int lp, int r, int k, int& p, int& q) {
  const int m = lp - 1;
  if (k == 0) {
    p = r;
    q = m;
  } else {
    p = (r + k) % m;
    q = (r - k + m) % m;
  }
  if (p > q) {
    int t = p;
    p = q;
    q = t;
  }
}

// Rotation (c, s) that zeroes A_pq (Golub & Van Loan, symmetric Schur decomposition of a 2x2).
__global__ void k_angles(int lp, int r, const double* __restrict__ A, double* __restrict__ rot,
                         int* __restrict__ pairs) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= lp / 2) return;
  int p, q;
  round_pair(lp, r, k, p, q);
  const double apq = A[(size_t)p * lp + q];
  double c = 1.0, s = 0.0;
  if (apq != 0.0) {
    const double app = A[(size_t)p * lp + p], aqq = A[(size_t)q * lp + q];
    const double tau = (aqq - app) / (2.0 * apq);
    double t;
    if (fabs(tau) > 1e150) t = 0.5 / tau;
    else t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
    c = 1.0 / sqrt(1.0 + t * t);
    s = t * c;
  }
  rot[2 * k] = c;
  rot[2 * k + 1] = s;
  pairs[2 * k] = p;
  pairs[2 * k + 1] = q;
}

// A <- J^T A J on every 2x2 block (pair a, pair b), b >= a, mirrored; V <- V J.
// Blocks [0, nA) of the grid do A (2D tiles of 16 x 16 pair-blocks), the rest do V.
__global__ void k_rotate(int lp, int l, int nApb, double* __restrict__ A, double* __restrict__ V,
                         const double* __restrict__ rot, const int* __restrict__ pairs, int nAblk) {
  const int half = lp / 2;
  if ((int)blockIdx.x < nAblk) {
    const int tilesPerRow = nApb;
    const int ta = blockIdx.x / tilesPerRow, tb = blockIdx.x % tilesPerRow;
    if (tb < ta) return;
    const int a = ta * 16 + threadIdx.y, b = tb * 16 + threadIdx.x;
    if (a >= half || b >= half || b < a) return;
    const int pa = pairs[2 * a], qa = pairs[2 * a + 1], pb = pairs[2 * b], qb = pairs[2 * b + 1];
    const double ca = rot[2 * a], sa = rot[2 * a + 1], cb = rot[2 * b], sb = rot[2 * b + 1];
    const double m00 = A[(size_t)pa * lp + pb], m01 = A[(size_t)pa * lp + qb];
    const double m10 = A[(size_t)qa * lp + pb], m11 = A[(size_t)qa * lp + qb];
    // rows: p' = c p - s q ; q' = s p + c q
    const double r00 = ca * m00 - sa * m10, r01 = ca * m01 - sa * m11;
    const double r10 = sa * m00 + ca * m10, r11 = sa * m01 + ca * m11;
    // columns: same map on the right
    double n00 = cb * r00 - sb * r01, n01 = sb * r00 + cb * r01;
    double n10 = cb * r10 - sb * r11, n11 = sb * r10 + cb * r11;
    if (a == b) {
      n01 = 0.0;   // the rotation zeroes this entry by construction
      A[(size_t)pa * lp + pa] = n00;
      A[(size_t)qa * lp + qa] = n11;
      A[(size_t)pa * lp + qa] = 0.0;
      A[(size_t)qa * lp + pa] = 0.0;
      return;
    }
    A[(size_t)pa * lp + pb] = n00;
    A[(size_t)pa * lp + qb] = n01;
    A[(size_t)qa * lp + pb] = n10;
    A[(size_t)qa * lp + qb] = n11;
    A[(size_t)pb * lp + pa] = n00;
    A[(size_t)qb * lp + pa] = n01;
    A[(size_t)pb * lp + qa] = n10;
    A[(size_t)qb * lp + qa] = n11;
  } else {
    // V: thread per (row i, pair b)
    const size_t idx = (size_t)(blockIdx.x - nAblk) * 256 + threadIdx.y * 16 + threadIdx.x;
    const size_t total = (size_t)l * half;
    if (idx >= total) return;
    const int i = (int)(idx / half), b = (int)(idx % half);
    const int pb = pairs[2 * b], qb = pairs[2 * b + 1];
    const double cb = rot[2 * b], sb = rot[2 * b + 1];
    if (sb == 0.0 && cb == 1.0) return;
    double* row = V + (size_t)i * lp;
    const double vp = row[pb], vq = row[qb];
    row[pb] = cb * vp - sb * vq;
    row[qb] = sb * vp + cb * vq;
  }
}

__global__ void k_offdiag_sumsq(int lp, const double* __restrict__ A, double* __restrict__ partial) {
  __shared__ double sh[256];
  double acc = 0.0;
  const size_t n = (size_t)lp * lp;
  for (size_t e = blockIdx.x * 256 + threadIdx.x; e < n; e += (size_t)gridDim.x * 256) {
    int i = (int)(e / lp), j = (int)(e % lp);
    if (i != j) acc = fma(A[e], A[e], acc);
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

__global__ void k_sum2(int nb, const double* __restrict__ partial, double* __restrict__ out) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nb; i += 256) acc += partial[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

// Place Z (l x l, ld l) into A (lp x lp) with a zero pad row/column; V = identity (or warm).
__global__ void k_init_pad(int l, int lp, double* __restrict__ A, double* __restrict__ V,
                           const double* __restrict__ Z, const double* __restrict__ warm) {
  const int j = blockIdx.x * 32 + threadIdx.x, i = blockIdx.y * 8 + threadIdx.y;
  if (i >= lp || j >= lp) return;
  if (Z) A[(size_t)i * lp + j] = (i < l && j < l) ? Z[(size_t)i * l + j] : 0.0;
  else if (i >= l || j >= l) A[(size_t)i * lp + j] = 0.0;
  double v;
  if (i < l && j < l) v = warm ? warm[(size_t)i * l + j] : (i == j ? 1.0 : 0.0);
  else v = (i == j) ? 1.0 : 0.0;
  V[(size_t)i * lp + j] = v;
}

// rank_i = #{ j : d_j < d_i or (d_j == d_i and j < i) }  (stable ascending order)
__global__ void k_rank(int l, int lp, const double* __restrict__ A, int* __restrict__ rank) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= l) return;
  const double di = A[(size_t)i * lp + i];
  int r = 0;
  for (int j = 0; j < l; ++j) {
    const double dj = A[(size_t)j * lp + j];
    r += (dj < di) || (dj == di && j < i);
  }
  rank[i] = r;
}

__global__ void k_gather(int l, int lp, const double* __restrict__ A, const double* __restrict__ V,
                         const int* __restrict__ rank, double* __restrict__ P,
                         double* __restrict__ sig) {
  const int j = blockIdx.x * 32 + threadIdx.x, i = blockIdx.y * 8 + threadIdx.y;
  if (i >= l || j >= l) return;
  const int rj = rank[j];
  P[(size_t)i * l + rj] = V[(size_t)i * lp + j];
  if (i == 0) sig[rj] = A[(size_t)j * lp + j];
}

}  // namespace

int eig_sym_f64(cudaStream_t st, int l, const double* Z, const double* warm, double* P,
                double* sig, JacobiWork& w, int max_sweeps, double* host_scal) {
  const int lp = std::max(2, l + (l & 1));   // even, >= 2
  const int half = lp / 2;
  w.A.alloc((size_t)lp * lp);
  w.V.alloc((size_t)lp * lp);
  w.rot.alloc((size_t)lp);
  w.pairs.alloc((size_t)lp);
  w.rank.alloc((size_t)l);
  w.partial.alloc(kReduceBlocks);
  w.scal.alloc(4);
  dim3 g2(cdiv(lp, 32), cdiv(lp, 8)), b2(32, 8);
  if (warm) {
    // A = warm^T Z warm: first V(:, :l) = Z warm (ld lp), then A = warm^T V
    gemm_f64(st, false, false, l, l, l, 1.0, Z, l, warm, l, nullptr, 0.0, w.V.p, lp, 0);
    gemm_f64(st, true, false, l, l, l, 1.0, warm, l, w.V.p, lp, nullptr, 0.0, w.A.p, lp, G_SYM);
    k_init_pad<<<g2, b2, 0, st>>>(l, lp, w.A.p, w.V.p, nullptr, warm);
  } else {
    k_init_pad<<<g2, b2, 0, st>>>(l, lp, w.A.p, w.V.p, Z, nullptr);
  }
  KOT_CHECK_LAUNCH();
  // ||A||_F^2 for the stopping test
  sumsq_f64(st, (size_t)lp * lp, w.A.p, w.scal.p + 1, w.partial.p);
  const int nApb = cdiv(half, 16);
  const int nAblk = nApb * nApb;
  const int nVblk = cdiv((size_t)l * half, 256);
  int sweeps = 0;
  double prev_off = INFINITY;
  for (; sweeps <= max_sweeps; ++sweeps) {
    k_offdiag_sumsq<<<kReduceBlocks, 256, 0, st>>>(lp, w.A.p, w.partial.p);
    k_sum2<<<1, 256, 0, st>>>(kReduceBlocks, w.partial.p, w.scal.p);
    KOT_LAUNCHED(2);
    KOT_CUDA(cudaMemcpyAsync(host_scal, w.scal.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    KOT_CUDA(cudaStreamSynchronize(st));
    const double off = std::sqrt(host_scal[0]), nrm = std::sqrt(host_scal[1]);
    if (!std::isfinite(off)) throw Error{KOT_ERR_NONFINITE, "eig: non-finite matrix"};
    if (off <= 1e-14 * nrm || nrm == 0.0) break;
    if (sweeps >= 2 && off > 0.5 * prev_off && off <= 1e-12 * nrm) break;   // at rounding floor
    if (sweeps == max_sweeps) throw Error{KOT_ERR_NO_CONVERGENCE, "eig: Jacobi did not converge"};
    prev_off = off;
    // algorithmic work of one round: 24 flops per rotated 2x2 block of A (upper half of the
    // half x half block grid), 6 per (row, pair) of V; bytes: each touched double read + written
    const double hb = (double)half * (half + 1) / 2.0;
    const double rflops = 24.0 * hb + 6.0 * (double)l * half;
    const double rbytes = 16.0 * (4.0 * hb + 4.0 * hb) + 16.0 * 2.0 * (double)l * half;
    for (int r = 0; r < lp - 1; ++r) {
      {
        ProfScope ps(st, KC_JACOBI_ANGLES, 0.0, 16.0 * 3 * half);
        k_angles<<<cdiv(half, 128), 128, 0, st>>>(lp, r, w.A.p, w.rot.p, w.pairs.p);
      }
      ProfScope ps(st, KC_JACOBI_ROTATE, rflops, rbytes);
      k_rotate<<<nAblk + nVblk, dim3(16, 16), 0, st>>>(lp, l, nApb, w.A.p, w.V.p, w.rot.p, w.pairs.p, nAblk);
    }
    KOT_LAUNCHED(2 * (lp - 1));
  }
  k_rank<<<cdiv(l, 128), 128, 0, st>>>(l, lp, w.A.p, w.rank.p);
  k_gather<<<dim3(cdiv(l, 32), cdiv(l, 8)), b2, 0, st>>>(l, lp, w.A.p, w.V.p, w.rank.p, P, sig);
  KOT_LAUNCHED(2);
  return sweeps;
}

}  // namespace kot
