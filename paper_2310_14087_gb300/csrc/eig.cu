// Symmetric eigen-decomposition by parallel cyclic two-sided Jacobi (textbook method: each
// rotation zeroes one off-diagonal pair, Golub & Van Loan's symmetric Schur 2 x 2 step), with
// round-robin ordering so that every round rotates lp/2 disjoint index pairs at once.
//
// Why Jacobi on this GPU: it needs no sequential scalar chain (no tridiagonal QR sweeps), it is
// exact for clustered and repeated eigenvalues (Z = -lambda1 I at the start of the solve), and it
// takes a warm start: the SSN iteration hands in the eigenbasis of the previous, nearby Z, so
// P^T Z P is already nearly diagonal and one or two sweeps finish the job.
//
// Each round updates every 2 x 2 block {p_a, q_a} x {p_b, q_b} of A (one thread per block, the
// blocks are disjoint) and every row of V on the rotated columns; the rotation of each pair is
// the textbook 2 x 2 symmetric Schur step (Golub & Van Loan) that zeroes A_pq.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "kot_internal.cuh"

namespace kot {

namespace {

inline int cdiv(size_t a, int b) { return (int)((a + b - 1) / b); }

// Round-robin (circle method) pairing of lp indices: round r in [0, lp-1), slot k in [0, lp/2).
// Slot 0 pairs r with lp - 1; slot k > 0 pairs (r + k) mod m with (r - k) mod m, m = lp - 1.
__device__ __forceinline__ void round_pair(int lp, int r, int k, int& p, int& q) {
  const int m = lp - 1;
  if (k == 0) {
    p = r;
    q = m;
  } else {
    p = r + k;
    if (p >= m) p -= m;
    q = r - k;
    if (q < 0) q += m;
  }
  if (p > q) {
    const int t = p;
    p = q;
    q = t;
  }
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

// Order-preserving integer key of a double (-0 and +0 share the key of +0): x < y iff key(x) <
// key(y) for non-NaN x, y.  Comparing keys costs integer instructions; FP64 compares would run
// on this part's scarce FP64 pipe.
__device__ __forceinline__ unsigned long long order_key(double x) {
  const unsigned long long b = (x == 0.0) ? 0ull : (unsigned long long)__double_as_longlong(x);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// rank_i = #{ j : d_j < d_i or (d_j == d_i and j < i) }  (stable ascending order); d_j is read
// with stride `stride` from `d` (the diagonal of A: stride lp + 1).  Block (32, 8): 32 values i
// per block, the 8 thread rows split the j range; keys are staged through shared memory.
__global__ void k_rank_stride(int l, const double* __restrict__ d, int stride, int* __restrict__ rank) {
  __shared__ unsigned long long sh[256];
  __shared__ int cnt[8][33];
  const int tx = threadIdx.x, ty = threadIdx.y, t = ty * 32 + tx;
  const int i = blockIdx.x * 32 + tx;
  const unsigned long long ki = i < l ? order_key(d[(size_t)i * stride]) : 0ull;
  int r = 0;
  for (int j0 = 0; j0 < l; j0 += 256) {
    __syncthreads();
    if (j0 + t < l) sh[t] = order_key(d[(size_t)(j0 + t) * stride]);
    __syncthreads();
    const int n = min(256, l - j0);
    for (int q = ty; q < n; q += 8) {
      const unsigned long long kj = sh[q];
      r += (kj < ki) || (kj == ki && j0 + q < i);
    }
  }
  cnt[ty][tx] = r;
  __syncthreads();
  if (ty == 0 && i < l) {
    int tot = 0;
#pragma unroll
    for (int y = 0; y < 8; ++y) tot += cnt[y][tx];
    rank[i] = tot;
  }
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

// ------------------------------------------------------------------ refinement of a warm basis
// One step of the iterative refinement of Ogita and Aishima (Japan J. Indust. Appl. Math. 35,
// 2018) for an approximate eigenbasis X of Z.  Writing X = X*(I + D) with X* an exact eigenbasis,
// G = X^T X ~ I + D + D^T and S = X^T Z X ~ L + D^T L + L D to first order, so
//   lam_i = S_ii / G_ii,   E_ii = (1 - G_ii) / 2,   E_ij = (S_ij - lam_j G_ij) / (lam_j - lam_i)
// gives E ~ -D and X (I + E) is an eigenbasis up to O(|D|^2): both the off-diagonal of the
// rotated Z and the loss of orthogonality shrink quadratically.  This kernel writes F = I + E,
// lam, and the largest |E_ij| (i != j) and |delta_ij - G_ij| as ordered bit patterns (a non-finite
// E orders above every finite value, so it always reads as "not converged").
__global__ void k_refine_correction(int l, int ld, const double* __restrict__ S, const double* __restrict__ G,
                                    double* __restrict__ F, double* __restrict__ lam,
                                    unsigned long long* __restrict__ mx) {
  pdl_wait();
  pdl_trigger();
  const int j = blockIdx.x * 32 + threadIdx.x, i = blockIdx.y * 8 + threadIdx.y;
  // lam_k = S_kk / G_kk for the block's 32 columns and 8 rows, one division each
  __shared__ double lcol[32], lrow[8];
  if (threadIdx.y == 0 && j < l) lcol[threadIdx.x] = S[(size_t)j * ld + j] / G[(size_t)j * ld + j];
  if (threadIdx.y == 1 && threadIdx.x < 8) {
    const int ii = blockIdx.y * 8 + threadIdx.x;
    if (ii < l) lrow[threadIdx.x] = S[(size_t)ii * ld + ii] / G[(size_t)ii * ld + ii];
  }
  __syncthreads();
  double e_abs = 0.0, r_abs = 0.0;
  if (i < l && j < l) {
    const size_t ij = (size_t)i * ld + j;
    const double g = G[ij];
    const double lj = lcol[threadIdx.x];
    double f;
    if (i == j) {
      f = 1.0 + 0.5 * (1.0 - g);
      r_abs = fabs(1.0 - g);
      lam[j] = lj;
      if (lj <= 0.0) atomicAdd(mx + 2, 1ull);   // |alpha-bar| if this step is the last
    } else {
      const double li = lrow[threadIdx.y];
      f = (S[ij] - lj * g) / (lj - li);
      e_abs = fabs(f);
      r_abs = fabs(g);
      if (!(e_abs <= 1e300)) e_abs = INFINITY;   // 0/0 or x/0: never converged
    }
    F[(size_t)i * l + j] = f;
  }
  // block maxima (non-negative doubles order like their bit patterns)
  __shared__ unsigned long long sm[2][8];
  unsigned long long be = (unsigned long long)__double_as_longlong(e_abs);
  unsigned long long br = (unsigned long long)__double_as_longlong(r_abs);
  for (int o = 16; o > 0; o >>= 1) {
    be = max(be, __shfl_xor_sync(0xffffffffu, be, o));
    br = max(br, __shfl_xor_sync(0xffffffffu, br, o));
  }
  if (threadIdx.x == 0) {
    sm[0][threadIdx.y] = be;
    sm[1][threadIdx.y] = br;
  }
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    for (int y = 1; y < 8; ++y) {
      be = max(be, sm[0][y]);
      br = max(br, sm[1][y]);
    }
    atomicMax(mx, be);
    atomicMax(mx + 1, br);
  }
}

__global__ void k_gather_vec(int l, const double* __restrict__ lam, const double* __restrict__ X, int ldx,
                             const int* __restrict__ rank, double* __restrict__ P,
                             double* __restrict__ sig) {
  const int j = blockIdx.x * 32 + threadIdx.x, i = blockIdx.y * 8 + threadIdx.y;
  if (i >= l || j >= l) return;
  const int rj = rank[j];
  P[(size_t)i * l + rj] = X[(size_t)i * ldx + j];
  if (i == 0) sig[rj] = lam[j];
}


// ------------------------------------------------------------------ persistent variant
// One cooperative launch runs every sweep.  Round r reads A_src and writes A_dst (double
// buffer), updates V in place, and -- from A_src and the round-r angles alone -- computes the
// round-(r+1) angles, so a single grid barrier separates rounds.  Cross-CTA data are read with
// ld.global.cg (L2), and the barrier gives up after a bounded number of polls (error flag).

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

constexpr long long kBarrierPolls = 40000000;   // polls (>= 32 ns apart after the first 1024)

__device__ __forceinline__ unsigned atom_add_acqrel_u32(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

// Grid-wide barrier for a cooperative launch.  bar[0] counts arrivals and bar[1] holds the last
// completed epoch; both are zeroed by the host before the launch and only grow, so there is no
// reset race.  Arrival is one acquire-release atomic per CTA (it publishes the CTA's writes,
// ordered before it by __syncthreads); the last arriver, which sees count == epoch * nblocks,
// publishes the epoch with one release store.  (Measured on GB300 at 152 CTAs: ~2.4 us; one
// release store per CTA flag costs ~50 us, a fence plus relaxed per-CTA stores ~3.1 us.)
// Returns false (and sets *err) if the wait gave up.
__device__ bool grid_barrier(unsigned* bar, unsigned nblocks, unsigned& epoch, int* err) {
  __shared__ int ok;
  __syncthreads();
  ++epoch;
  if (threadIdx.x == 0) {
    ok = 1;
    const unsigned arrived = atom_add_acqrel_u32(bar, 1u) + 1u;
    if (arrived == epoch * nblocks) {
      st_release_u32(bar + 1, epoch);
    } else {
      long long polls = 0;
      while ((int)(ld_acquire_u32(bar + 1) - epoch) < 0) {
        if (++polls > kBarrierPolls) {
          atomicExch(err, 1);
          ok = 0;
          break;
        }
        if (polls > 1024) __nanosleep(32);
      }
    }
  }
  __syncthreads();
  return ok != 0;
}

template <typename T>
struct CoopArgs {
  int lp, l, max_sweeps;
  T* A0;
  T* A1;
  T* V;
  T* rot0;             // round-parity 0 angles (c, s) per pair
  T* rot1;
  double* partial;     // gridDim.x partial sums
  unsigned* bar;       // [count, generation]
  int* err;
  int* sweeps_out;
  double tol_rel;      // stop when off(A) <= tol_rel * ||A||_F
  double floor_rel;    // ... or when a sweep stalls (off > 0.5 prev) below floor_rel * ||A||_F
};

// Jacobi rotation (c, s) for the pair (p, q): the 2 x 2 symmetric Schur step.  The angle is
// computed in FP32 -- from the FP64 difference a_qq - a_pp, so nearly equal diagonal entries do
// not cancel -- which is ~10x shorter than the FP64 divide/square-root chain on this part; the
// pair (c, s) is then renormalised in FP64 (two Newton steps on c^2 + s^2 = 1), so every rotation
// is orthogonal to FP64 precision and A stays an exact similarity transform of Z.  The rotated
// entry is left at ~1e-7 |a_pq| instead of 0 and is removed by the next sweep.
template <typename T>
__device__ __forceinline__ void rot_angle(T app, T aqq, T apq, T& c, T& s) {
  c = T(1);
  s = T(0);
  const float fpq = (float)apq;
  const float fd = (float)(aqq - app);
  if (fpq == 0.0f || !(fabsf(fpq) > 1e-30f * fabsf(fd))) return;
  const float tau = fd / (2.0f * fpq);
  float t;
  if (fabsf(tau) > 1e18f) t = 0.5f / tau;
  else t = copysignf(1.0f, tau) / (fabsf(tau) + sqrtf(1.0f + tau * tau));
  const float fc = rsqrtf(1.0f + t * t);
  T c0 = (T)fc, s0 = (T)(t * fc);
#pragma unroll
  for (int i = 0; i < 2; ++i) {   // Newton steps on c^2 + s^2 = 1: 1e-7 -> 1e-14 -> rounding
    const T corr = T(1.5) - T(0.5) * (c0 * c0 + s0 * s0);
    c0 *= corr;
    s0 *= corr;
  }
  c = c0;
  s = s0;
}

// New 2x2 block J_a^T M J_b (rows p_a, q_a; columns p_b, q_b).
template <typename T>
__device__ __forceinline__ void rot_block(T ca, T sa, T cb, T sb, T m00, T m01, T m10, T m11,
                                          T& n00, T& n01, T& n10, T& n11) {
  const T r00 = ca * m00 - sa * m10, r01 = ca * m01 - sa * m11;
  const T r10 = sa * m00 + ca * m10, r11 = sa * m01 + ca * m11;
  n00 = cb * r00 - sb * r01;
  n01 = sb * r00 + cb * r01;
  n10 = cb * r10 - sb * r11;
  n11 = sb * r10 + cb * r11;
}

// Slot of the round-r pair that contains index i (inverse of round_pair).
__device__ __forceinline__ int slot_of(int lp, int r, int i) {
  const int m = lp - 1;
  if (i == m || i == r) return 0;
  int k = i - r;
  if (k < 0) k += m;
  if (k >= lp / 2) k = m - k;
  return k;
}

template <typename T>
__device__ double block_reduce_sum(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  double r = sh[0];
  __syncthreads();
  return r;
}

// Threads per CTA of the cooperative kernel (its "block size"): 256, 512 (default) or 1024,
// chosen per size bucket by the autotuner.
constexpr int kCoopThreads = 512;

template <typename T, int NT>
__global__ void __launch_bounds__(NT) k_jacobi_coop(CoopArgs<T> a) {
  __shared__ double sh[NT];
  const int lp = a.lp, l = a.l, half = lp / 2;
  const unsigned nb = gridDim.x;
  const size_t gtid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t gstride = (size_t)gridDim.x * blockDim.x;
  T* A[2] = {a.A0, a.A1};
  T* rot[2] = {a.rot0, a.rot1};
  int cur = 0;
  unsigned epoch = 0;   // barriers passed (identical in every CTA)

  // deterministic sum of a per-block partial over the grid (every block gets the same value)
  // (two halves of the partial array alternate, so a block still reading one sum's partials
  // never sees them overwritten by the next sum's)
  int sum_calls = 0;
  auto grid_sum = [&](double v, bool& ok) -> double {
    double* part = a.partial + (size_t)(sum_calls++ & 1) * nb;
    double bs = block_reduce_sum<T>(v, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = bs;
    ok = grid_barrier(a.bar, nb, epoch, a.err);
    double tot = 0.0;
    for (unsigned i = threadIdx.x; i < nb; i += blockDim.x) tot += __ldcg(part + i);
    tot = block_reduce_sum<T>(tot, sh);
    return tot;
  };

  // round-0 angles and ||A||_F^2
  double acc = 0.0;
  for (size_t e = gtid; e < (size_t)lp * lp; e += gstride) {
    const double v = (double)__ldcg(A[0] + e);
    acc += v * v;
  }
  for (size_t k = gtid; k < (size_t)half; k += gstride) {
    int p, q;
    round_pair(lp, 0, (int)k, p, q);
    T c, s;
    rot_angle<T>(__ldcg(A[0] + (size_t)p * lp + p), __ldcg(A[0] + (size_t)q * lp + q),
                 __ldcg(A[0] + (size_t)p * lp + q), c, s);
    rot[0][2 * k] = c;
    rot[0][2 * k + 1] = s;
  }
  bool ok = true;
  const double nrm2 = grid_sum(acc, ok);
  if (!ok) return;
  double prev_off = INFINITY;
  int sweep = 0;
  unsigned gr = 0;   // rounds executed so far: round gr uses angles rot[gr & 1]
  for (;; ++sweep) {
    // off-diagonal norm of the current A
    acc = 0.0;
    for (int e = (int)gtid; e < lp * lp; e += (int)gstride) {
      const int i = e / lp, j = e - i * lp;
      if (i != j) {
        const double v = (double)__ldcg(A[cur] + e);
        acc += v * v;
      }
    }
    const double off2 = grid_sum(acc, ok);
    if (!ok) return;
    const double off = sqrt(off2), nrm = sqrt(nrm2);
    if (!(off > a.tol_rel * nrm) || nrm == 0.0) break;
    if (sweep >= 2 && off > 0.5 * prev_off && off <= a.floor_rel * nrm) break;
    if (sweep >= a.max_sweeps) {
      if (gtid == 0) atomicExch(a.err, 2);       // not converged
      break;
    }
    prev_off = off;
    for (int r = 0; r < lp - 1; ++r) {
      const T* src = A[cur];
      T* dst = A[cur ^ 1];
      const T* rc = rot[gr & 1];
      T* rn = rot[(gr + 1) & 1];
      const int rnext = (r + 1 == lp - 1) ? 0 : r + 1;
      const int nAu = half * (half + 1) / 2, nV = l * half, nN = half;
      // The round's items: the 2 x 2 blocks (ia, ib >= ia) of A, the (row, pair) items of V and
      // the next round's angles.  A and V items are taken contiguously along the grid (row by
      // row, so the lanes of a warp touch neighbouring columns); the angle items are dealt
      // round-robin over the CTAs (item k -> CTA k mod grid, thread k / grid): a few FP64
      // divide/square-root chains per SM instead of all of them on the one or two SMs a
      // contiguous range would land on (FP64 issues ~2 ops/clk per SM).
      for (int k = (int)(threadIdx.x * nb + blockIdx.x); k < nN; k += (int)gstride) {
          // angle of next-round pair k from the values this round writes, recomputed here
          int pn, qn;
          round_pair(lp, rnext, k, pn, qn);
          const int sp = slot_of(lp, r, pn), sq = slot_of(lp, r, qn);
          int pp, qp, pq_, qq;
          round_pair(lp, r, sp, pp, qp);
          round_pair(lp, r, sq, pq_, qq);
          const T cp = __ldcg(rc + 2 * sp), spn = __ldcg(rc + 2 * sp + 1);
          const T cq = __ldcg(rc + 2 * sq), sqn = __ldcg(rc + 2 * sq + 1);
          // diagonal entries of pn and qn after this round
          T d00, d01, d10, d11, app, aqq, apq;
          rot_block<T>(cp, spn, cp, spn, __ldcg(src + (size_t)pp * lp + pp), __ldcg(src + (size_t)pp * lp + qp),
                       __ldcg(src + (size_t)qp * lp + pp), __ldcg(src + (size_t)qp * lp + qp), d00, d01, d10, d11);
          app = (pn == pp) ? d00 : d11;
          rot_block<T>(cq, sqn, cq, sqn, __ldcg(src + (size_t)pq_ * lp + pq_), __ldcg(src + (size_t)pq_ * lp + qq),
                       __ldcg(src + (size_t)qq * lp + pq_), __ldcg(src + (size_t)qq * lp + qq), d00, d01, d10, d11);
          aqq = (qn == pq_) ? d00 : d11;
          // off-diagonal entry (pn, qn): block (slot sp rows) x (slot sq columns)
          if (sp == sq) {
            apq = d01;   // never happens for round-robin pairings (consecutive rounds differ)
          } else {
            rot_block<T>(cp, spn, cq, sqn, __ldcg(src + (size_t)pp * lp + pq_), __ldcg(src + (size_t)pp * lp + qq),
                         __ldcg(src + (size_t)qp * lp + pq_), __ldcg(src + (size_t)qp * lp + qq), d00, d01, d10, d11);
            apq = (pn == pp) ? ((qn == pq_) ? d00 : d01) : ((qn == pq_) ? d10 : d11);
          }
          T c, s;
          rot_angle<T>(app, aqq, apq, c, s);
          rn[2 * k] = c;
          rn[2 * k + 1] = s;
      }
      for (size_t it = gtid; it < (size_t)nAu + nV; it += gstride) {
        if (it < (size_t)nAu) {
          // upper-triangle block index -> (ia, ib): row ia holds blocks ia .. half - 1 and starts
          // at ia half - ia (ia - 1)/2
          const int t = (int)it;
          const float bq = 2.0f * half + 1.0f;
          int ia = (int)((bq - sqrtf(fmaxf(bq * bq - 8.0f * t, 0.0f))) * 0.5f);
          if (ia < 0) ia = 0;
          while (ia > 0 && ia * half - ia * (ia - 1) / 2 > t) --ia;
          while ((ia + 1) * half - (ia + 1) * ia / 2 <= t) ++ia;
          const int ib = ia + (t - (ia * half - ia * (ia - 1) / 2));
          int pa, qa, pb, qb;
          round_pair(lp, r, ia, pa, qa);
          round_pair(lp, r, ib, pb, qb);
          const T ca = __ldcg(rc + 2 * ia), sa = __ldcg(rc + 2 * ia + 1);
          const T cb = __ldcg(rc + 2 * ib), sb = __ldcg(rc + 2 * ib + 1);
          T n00, n01, n10, n11;
          rot_block<T>(ca, sa, cb, sb, __ldcg(src + (size_t)pa * lp + pb), __ldcg(src + (size_t)pa * lp + qb),
                       __ldcg(src + (size_t)qa * lp + pb), __ldcg(src + (size_t)qa * lp + qb),
                       n00, n01, n10, n11);
          if (ia == ib) {
            dst[(size_t)pa * lp + pa] = n00;
            dst[(size_t)qa * lp + qa] = n11;
            dst[(size_t)pa * lp + qa] = n01;
            dst[(size_t)qa * lp + pa] = n01;
          } else {
            dst[(size_t)pa * lp + pb] = n00;
            dst[(size_t)pa * lp + qb] = n01;
            dst[(size_t)qa * lp + pb] = n10;
            dst[(size_t)qa * lp + qb] = n11;
            dst[(size_t)pb * lp + pa] = n00;
            dst[(size_t)qb * lp + pa] = n01;
            dst[(size_t)pb * lp + qa] = n10;
            dst[(size_t)qb * lp + qa] = n11;
          }
        } else {
          const int v = (int)(it - nAu);
          const int i = v / half, b = v - i * half;
          int pb, qb;
          round_pair(lp, r, b, pb, qb);
          const T cb = __ldcg(rc + 2 * b), sb = __ldcg(rc + 2 * b + 1);
          if (!(sb == T(0) && cb == T(1))) {
          T* row = a.V + (size_t)i * lp;
          const T vp = __ldcg(row + pb), vq = __ldcg(row + qb);
          row[pb] = cb * vp - sb * vq;
          row[qb] = sb * vp + cb * vq;
          }
        }
      }
      if (!grid_barrier(a.bar, nb, epoch, a.err)) return;
      cur ^= 1;
      ++gr;
    }
  }
  if (gtid == 0) a.sweeps_out[0] = sweep * 2 + cur;   // sweeps and the buffer holding A
}
}  // namespace

int jacobi_sym_f64(cudaStream_t st, int l, const double* Z, const double* warm, double* P,
                   double* sig, JacobiWork& w, int max_sweeps, double* host_scal, int ctas);

namespace {

// Refinement thresholds on max |E_ij| (and on the loss of orthogonality max |I - X^T X|): a
// first correction above kRefineStart means the warm basis is too far for the iteration (or a
// pair is degenerate), and a later one that is not below kRefineContract times its predecessor
// means it is not converging; either way Jacobi takes over.  Converging steps contract the error
// about quadratically (0.4 -> 0.16 -> 0.03 -> 1e-3), so a start of a few tenths still finishes in
// the step budget at a fraction of the cost of Jacobi sweeps.  At or below w.refine_done (1e-8
// unless the caller asks otherwise) the step just taken leaves an error of order refine_done^2,
// so it is the last.
constexpr double kRefineStart = 0.5;
constexpr double kRefineContract = 0.5;

// Refine the warm basis into P, sig (ascending).  Returns the steps taken, or 0 if the iteration
// gave up (P and sig are then untouched).
int refine_sym_f64(cudaStream_t st, int l, const double* Z, const double* warm, double* P,
                   double* sig, JacobiWork& w, int max_steps, double prev_me0 = 0.0) {
  const size_t L2 = (size_t)l * l;
  // FP64 pipes: five products per step, the two symmetric ones on their upper halves only.
  // Emulated FP64 (w.oz): the basis X sits in the right half of an l x 2l buffer whose left half
  // holds Y = Z X, so that X^T [Y | X] gives S and G in one product (launches, not flops, are
  // what a step costs at moderate l).  Read as 2l x l rows, the buffer interleaves the rows of Y
  // and X, so one product [Y | X] (I + E) both updates the basis and carries Y = Z X to it: only
  // the first step multiplies by Z, each step after it takes two products.
  const bool merged = w.oz != nullptr;
  const int ldx = merged ? 2 * l : l;
  for (DevBuf<double>* b : {&w.Xa, &w.Xb, &w.S}) b->alloc(merged ? 2 * L2 : L2);
  for (DevBuf<double>* b : {&w.Y, &w.G, &w.F}) b->alloc(L2);
  w.lam.alloc((size_t)l);
  w.rank.alloc((size_t)l);
  w.mx.alloc(3);
  const dim3 g2(cdiv(l, 32), cdiv(l, 8)), b2(32, 8);
  const double* X = warm;
  int ldX = l;
  if (merged) {
    copy_mat(st, l, l, warm, l, w.Xa.p + l, ldx);
    X = w.Xa.p + l;
    ldX = ldx;
  }
  double prev_me = prev_me0;
  for (int k = 0; k < max_steps; ++k) {
    const double* S;
    const double* G;
    int lds;
    double* Xn;
    if (merged) {
      double* B = (k & 1) ? w.Xb.p : w.Xa.p;            // [Z X | X], X = B + l
      Xn = ((k & 1) ? w.Xa.p : w.Xb.p) + l;
      if (k == 0) gemm_acc(st, w.oz, false, false, l, l, l, 1.0, Z, l, X, ldX, nullptr, 0.0, B, ldx, 0);
      gemm_acc(st, w.oz, true, false, l, 2 * l, l, 1.0, X, ldX, B, ldx, nullptr, 0.0, w.S.p, ldx, 0);
      S = w.S.p;                                          // X^T Z X
      G = w.S.p + l;                                      // X^T X
      lds = ldx;
    } else {
      Xn = (k & 1) ? w.Xb.p : w.Xa.p;
      gemm_acc(st, w.oz, false, false, l, l, l, 1.0, Z, l, X, ldX, nullptr, 0.0, w.Y.p, l, 0);       // Y = Z X
      gemm_acc(st, w.oz, true, false, l, l, l, 1.0, X, ldX, w.Y.p, l, nullptr, 0.0, w.S.p, l, G_SYM); // S = X^T Y
      gemm_acc(st, w.oz, true, false, l, l, l, 1.0, X, ldX, X, ldX, nullptr, 0.0, w.G.p, l, G_SYM);   // G = X^T X
      S = w.S.p;
      G = w.G.p;
      lds = l;
    }
    KOT_CUDA(cudaMemsetAsync(w.mx.p, 0, 3 * sizeof(unsigned long long), st));
    {
      ProfScope ps(st, KC_REFINE, 12.0 * (double)L2, 8.0 * 3.0 * (double)L2);
      launch_pdl(k_refine_correction, dim3(g2), dim3(b2), 0, st, l, lds, S, G, w.F.p, w.lam.p, w.mx.p);
      KOT_CHECK_LAUNCH();
      KOT_LAUNCHED(1);
    }
    if (merged)   // [Y | X] (I + E): rows (Y_i, X_i) of the buffer as 2l rows of length l
      gemm_acc(st, w.oz, false, false, 2 * l, l, l, 1.0, X - l, l, w.F.p, l, nullptr, 0.0, Xn - l, l, 0);
    else
      gemm_acc(st, w.oz, false, false, l, l, l, 1.0, X, ldX, w.F.p, l, nullptr, 0.0, Xn, ldx, 0);   // X (I + E)
    unsigned long long hm[3] = {0, 0, 0};
    KOT_CUDA(cudaMemcpyAsync(hm, w.mx.p, sizeof(hm), cudaMemcpyDeviceToHost, st));
    KOT_CUDA(cudaStreamSynchronize(st));
    double me, mr;
    std::memcpy(&me, &hm[0], sizeof(double));
    std::memcpy(&mr, &hm[1], sizeof(double));
    const double cap = (k == 0 && prev_me <= 0.0) ? kRefineStart : kRefineContract * prev_me;
    if (!(me <= cap) || !(mr <= kRefineStart)) return 0;
    prev_me = me;
    X = Xn;
    ldX = ldx;
    if (me <= w.refine_done && mr <= w.refine_done) {
      k_rank_stride<<<cdiv(l, 32), dim3(32, 8), 0, st>>>(l, w.lam.p, 1, w.rank.p);
      k_gather_vec<<<g2, b2, 0, st>>>(l, w.lam.p, X, ldX, w.rank.p, P, sig);
      KOT_CHECK_LAUNCH();
      KOT_LAUNCHED(2);
      w.last_nb = (int)hm[2];
      return k + 1;
    }
  }
  return 0;
}

// Refinement without a warm basis, from the identity: its first step needs no product (S = Z,
// G = I), so a Z that is diagonal to the tolerance, or too far from diagonal, costs one small
// kernel and a readback; otherwise X = I + E continues through refine_sym_f64.  Returns the
// steps (0: gave up); *diag = the first correction already met the tolerance (Z is diagonal,
// the basis is the identity up to the sort).
int refine_from_identity(cudaStream_t st, int l, const double* Z, double* P, double* sig,
                         JacobiWork& w, int max_steps, bool* diag) {
  *diag = false;
  const size_t L2 = (size_t)l * l;
  if (w.eye_l != l) {
    w.eye.alloc(L2);
    fill(st, L2, 0.0, w.eye.p);
    add_diag(st, l, 1.0, w.eye.p, l);
    w.eye_l = l;
  }
  w.F.alloc(L2);
  w.lam.alloc((size_t)l);
  w.rank.alloc((size_t)l);
  w.mx.alloc(3);
  KOT_CUDA(cudaMemsetAsync(w.mx.p, 0, 3 * sizeof(unsigned long long), st));
  const dim3 g2(cdiv(l, 32), cdiv(l, 8)), b2(32, 8);
  {
    ProfScope ps(st, KC_REFINE, 12.0 * (double)L2, 8.0 * 3.0 * (double)L2);
    launch_pdl(k_refine_correction, dim3(g2), dim3(b2), 0, st, l, l, Z, (const double*)w.eye.p, w.F.p,
               w.lam.p, w.mx.p);
    KOT_CHECK_LAUNCH();
    KOT_LAUNCHED(1);
  }
  unsigned long long hm[3] = {0, 0, 0};
  KOT_CUDA(cudaMemcpyAsync(hm, w.mx.p, sizeof(hm), cudaMemcpyDeviceToHost, st));
  KOT_CUDA(cudaStreamSynchronize(st));
  double me;
  std::memcpy(&me, &hm[0], sizeof(double));
  if (!(me <= kRefineStart)) return 0;
  if (me <= w.refine_done) {   // X = I + E with |E| <= refine_done: the last step
    k_rank_stride<<<cdiv(l, 32), dim3(32, 8), 0, st>>>(l, w.lam.p, 1, w.rank.p);
    k_gather_vec<<<g2, b2, 0, st>>>(l, w.lam.p, w.F.p, l, w.rank.p, P, sig);
    KOT_CHECK_LAUNCH();
    KOT_LAUNCHED(2);
    w.last_nb = (int)hm[2];
    *diag = true;
    return 1;
  }
  if (max_steps < 2) return 0;
  // continue from X = I + E (F is overwritten by the next correction, so it is copied first)
  w.X0.alloc(L2);
  copy_mat(st, l, l, w.F.p, l, w.X0.p, l);
  const int k = refine_sym_f64(st, l, Z, w.X0.p, P, sig, w, max_steps - 1, me);
  return k > 0 ? k + 1 : 0;
}

// ------------------------------------------------------------------ shared-memory FP32 Jacobi
// Cold decompositions of small matrices (l <= kSmemJacobiMax): one CTA per matrix holds A and V in
// FP32 in shared memory and runs parallel cyclic two-sided Jacobi (round-robin pairs, every 2 x 2
// block of a round updated independently), synchronising with __syncthreads instead of a grid
// barrier and issuing on the FP32 pipes (64x the FP64 rate of this part).  The basis it returns is
// accurate to FP32 (orthogonality ~1e-6); the FP64 refinement takes it from there.
constexpr int kSmemJacobiMax = 160;
constexpr int kSmemJacobiSweeps = 20;
constexpr int kSmemJacobiThreads = 1024;

__global__ void __launch_bounds__(kSmemJacobiThreads, 1)
    k_jacobi_smem_f32(int l, const double* __restrict__ Z, double* __restrict__ Vout,
                      int* __restrict__ diag) {
  extern __shared__ float jsm[];
  const int lp = l + (l & 1), ld = lp + 1, np = lp / 2;
  const int nblk = np * (np + 1) / 2;      // pair blocks (P <= Q) of the upper triangle
  float* A = jsm;                          // lp x ld
  float* V = A + (size_t)lp * ld;          // lp x ld
  float* cs = V + (size_t)lp * ld;         // np x (c, s)
  int2* pq = reinterpret_cast<int2*>(cs + lp);          // np: the round's pairs
  ushort2* blk = reinterpret_cast<ushort2*>(pq + np);  // nblk: (pair index P, pair index Q)
  __shared__ float red[2][32];
  __shared__ int done;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < lp * lp; e += nt) {
    const int i = e / lp, j = e - i * lp;
    A[i * ld + j] = (i < l && j < l) ? (float)(0.5 * (Z[(size_t)i * l + j] + Z[(size_t)j * l + i])) : 0.0f;
    V[i * ld + j] = (i == j) ? 1.0f : 0.0f;
  }
  for (int b = tid; b < nblk; b += nt) {
    // block b of the upper triangle: row bi starts at bi np - bi (bi - 1) / 2
    const float tn = (float)(2 * np + 1);
    int bi = (int)(0.5f * (tn - sqrtf(tn * tn - 8.0f * (float)b)));
    bi = max(0, min(bi, np - 1));
    while (bi > 0 && bi * np - bi * (bi - 1) / 2 > b) --bi;
    while (bi + 1 < np && (bi + 1) * np - (bi + 1) * bi / 2 <= b) ++bi;
    blk[b] = make_ushort2((unsigned short)bi, (unsigned short)(bi + (b - (bi * np - bi * (bi - 1) / 2))));
  }
  if (tid == 0) done = 0;
  __syncthreads();
  {
    // an exactly diagonal Z (e.g. a multiple of I) is reported and left to the caller
    int nz = 0;
    for (int e = tid; e < lp * lp; e += nt) {
      const int i = e / lp, j = e - i * lp;
      nz |= (i != j && A[i * ld + j] != 0.0f);
    }
    nz = __syncthreads_or(nz);
    if (tid == 0) *diag = nz ? 0 : 1;
  }
  for (int sweep = 0; sweep < kSmemJacobiSweeps; ++sweep) {
    for (int r = 0; r < lp - 1; ++r) {
      // angles of the round's pairs (symmetric Schur 2 x 2, Rutishauser's update of the diagonal)
      if (tid < np) {
        int p, q;
        round_pair(lp, r, tid, p, q);
        const float app = A[p * ld + p], aqq = A[q * ld + q], apq = A[p * ld + q];
        float c = 1.0f, s = 0.0f;
        if (apq != 0.0f) {
          const float tau = (aqq - app) / (2.0f * apq);
          const float t = (tau >= 0.0f ? 1.0f : -1.0f) / (fabsf(tau) + sqrtf(1.0f + tau * tau));
          c = rsqrtf(1.0f + t * t);
          s = t * c;
        }
        cs[2 * tid] = c;
        cs[2 * tid + 1] = s;
        pq[tid] = make_int2(p, q);
      }
      __syncthreads();
      // A <- J^T A J on the blocks P <= Q (mirrored), V <- V J
      for (int b = tid; b < nblk; b += nt) {
        const ushort2 bq = blk[b];
        const int bi = bq.x, bj = bq.y;
        const int2 pa = pq[bi], pb = pq[bj];
        const int p1 = pa.x, q1 = pa.y, p2 = pb.x, q2 = pb.y;
        const float c1 = cs[2 * bi], s1 = cs[2 * bi + 1], c2 = cs[2 * bj], s2 = cs[2 * bj + 1];
        if (bi == bj) {
          const float app = A[p1 * ld + p1], aqq = A[q1 * ld + q1], apq = A[p1 * ld + q1];
          const float t = (c1 != 0.0f) ? s1 / c1 : 0.0f;
          A[p1 * ld + p1] = app - t * apq;
          A[q1 * ld + q1] = aqq + t * apq;
          A[p1 * ld + q1] = 0.0f;
          A[q1 * ld + p1] = 0.0f;
        } else {
          const float a11 = A[p1 * ld + p2], a12 = A[p1 * ld + q2];
          const float a21 = A[q1 * ld + p2], a22 = A[q1 * ld + q2];
          const float b11 = c2 * a11 - s2 * a12, b12 = s2 * a11 + c2 * a12;
          const float b21 = c2 * a21 - s2 * a22, b22 = s2 * a21 + c2 * a22;
          const float n11 = c1 * b11 - s1 * b21, n21 = s1 * b11 + c1 * b21;
          const float n12 = c1 * b12 - s1 * b22, n22 = s1 * b12 + c1 * b22;
          A[p1 * ld + p2] = n11;
          A[q1 * ld + p2] = n21;
          A[p1 * ld + q2] = n12;
          A[q1 * ld + q2] = n22;
          A[p2 * ld + p1] = n11;
          A[p2 * ld + q1] = n21;
          A[q2 * ld + p1] = n12;
          A[q2 * ld + q1] = n22;
        }
      }
      for (int e = tid; e < lp * np; e += nt) {
        const int i = e / np, k = e - i * np;
        const int2 pk = pq[k];
        const int p = pk.x, q = pk.y;
        const float c = cs[2 * k], s = cs[2 * k + 1];
        const float vp = V[i * ld + p], vq = V[i * ld + q];
        V[i * ld + p] = c * vp - s * vq;
        V[i * ld + q] = s * vp + c * vq;
      }
      __syncthreads();
    }
    // off-diagonal against total Frobenius mass: FP32 has converged near 1e-7
    float off = 0.0f, tot = 0.0f;
    for (int e = tid; e < lp * lp; e += nt) {
      const int i = e / lp, j = e - i * lp;
      const float a = A[i * ld + j];
      tot += a * a;
      if (i != j) off += a * a;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      tot += __shfl_xor_sync(0xffffffffu, tot, o);
    }
    if ((tid & 31) == 0) {
      red[0][tid >> 5] = off;
      red[1][tid >> 5] = tot;
    }
    __syncthreads();
    if (tid == 0) {
      float so = 0.0f, st = 0.0f;
      for (int w = 0; w < (nt >> 5); ++w) {
        so += red[0][w];
        st += red[1][w];
      }
      done = (so <= 4e-14f * st) ? 1 : 0;
    }
    __syncthreads();
    if (done) break;
  }
  for (int e = tid; e < l * l; e += nt) {
    const int i = e / l, j = e - i * l;
    Vout[(size_t)i * l + j] = (double)V[i * ld + j];
  }
}

// FP32 eigenbasis of Z (l <= kSmemJacobiMax) into B (l x l, FP64, row-major, column j = vector j);
// *diag (device) = 1 when Z was exactly diagonal.
void jacobi_smem_f32(cudaStream_t st, int l, const double* Z, double* B, int* diag) {
  const int lp = l + (l & 1);
  // A, V (lp x (lp + 1) floats each), angles (lp floats), pairs (lp / 2 int2), block table
  auto bytes = [](size_t lpv) {
    const size_t npv = lpv / 2;
    return (2 * lpv * (lpv + 1) + lpv) * sizeof(float) + npv * sizeof(int2) + npv * (npv + 1) / 2 * 4;
  };
  const size_t smem = bytes((size_t)lp);
  static bool attr[64] = {};
  int dev = 0;
  KOT_CUDA(cudaGetDevice(&dev));
  if (dev >= 0 && dev < 64 && !attr[dev]) {
    const size_t mx = bytes((size_t)kSmemJacobiMax);
    KOT_CUDA(cudaFuncSetAttribute(k_jacobi_smem_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx));
    attr[dev] = true;
  }
  k_jacobi_smem_f32<<<1, kSmemJacobiThreads, smem, st>>>(l, Z, B, diag);
  KOT_CHECK_LAUNCH();
}

}  // namespace

int eig_sym_f64(cudaStream_t st, int l, const double* Z, const double* warm, double* P,
                double* sig, JacobiWork& w, int max_sweeps, double* host_scal, int ctas,
                int max_refine, const double* warm2) {
  w.last_sweeps = 0;
  w.last_refine = 0;
  w.last_nb = -1;
  w.last_trivial = false;
  if (max_refine > 0) {
    // No basis at all: try the identity first.  A nearly diagonal Z (the first projections of a
    // solve when the Gram matrix K is close to diagonal, small bandwidths) refines from it in a
    // few products, where cold Jacobi sweeps cost l - 1 grid-synchronised rounds each.
    if (!warm && !warm2) {
      bool diag = false;
      const int k = refine_from_identity(st, l, Z, P, sig, w, max_refine, &diag);
      if (k > 0) {
        w.last_refine = k;
        w.last_trivial = diag;
        return 0;
      }
    }
    for (const double* start : {warm, warm2}) {
      if (!start) continue;
      const int k = refine_sym_f64(st, l, Z, start, P, sig, w, max_refine);
      if (k > 0) {
        w.last_refine = k;
        return 0;
      }
    }
  }
  // Still cold and small: an FP32 basis from the shared-memory Jacobi, refined to FP64 (or, where
  // the refinement gives up, e.g. inside tight eigenvalue clusters, the start of the FP64 sweeps).
  const double* start = warm;
  if (!warm && !warm2 && max_refine > 0 && l >= 2 && l <= kSmemJacobiMax) {
    w.B32.alloc((size_t)l * l);
    w.flags.alloc(2);
    jacobi_smem_f32(st, l, Z, w.B32.p, w.flags.p + 1);
    int hdiag = 0;
    KOT_CUDA(cudaMemcpyAsync(&hdiag, w.flags.p + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    KOT_CUDA(cudaStreamSynchronize(st));
    if (!hdiag) {
      const int k = refine_sym_f64(st, l, Z, w.B32.p, P, sig, w, max_refine);
      if (k > 0) {
        w.last_refine = k;
        return 0;
      }
      // Jacobi from a warm basis needs orthonormal columns: two Newton-Schulz steps
      // B <- B (3 I - B^T B) / 2 take the FP32 basis's ~1e-6 loss of orthogonality to FP64 rounding
      const size_t L2 = (size_t)l * l;
      w.G.alloc(L2);
      w.F.alloc(L2);
      w.X0.alloc(L2);
      double* b0 = w.B32.p;
      double* b1 = w.X0.p;
      for (int it = 0; it < 2; ++it) {
        gemm_acc(st, w.oz, true, false, l, l, l, 1.0, b0, l, b0, l, nullptr, 0.0, w.G.p, l, G_SYM);
        axpby(st, L2, -0.5, w.G.p, 0.0, nullptr, w.F.p);
        add_diag(st, l, 1.5, w.F.p, l);
        gemm_acc(st, w.oz, false, false, l, l, l, 1.0, b0, l, w.F.p, l, nullptr, 0.0, b1, l, 0);
        std::swap(b0, b1);
      }
      start = b0;
    }
  }
  w.last_sweeps = jacobi_sym_f64(st, l, Z, start, P, sig, w, max_sweeps, host_scal, ctas);
  w.last_trivial = !start && w.last_sweeps == 0;
  return w.last_sweeps;
}

namespace {
int g_tuned_ctas[64][32] = {};
int g_tuned_threads[64][32] = {};
int l_bucket(int l) {
  int b = 0;
  while ((1 << b) < l && b < 31) ++b;
  return b;
}
}  // namespace

int tuned_jacobi_ctas(int dev, int l) {
  if (dev < 0 || dev >= 64) return 0;
  return g_tuned_ctas[dev][l_bucket(l)];
}

void set_tuned_jacobi_ctas(int dev, int l, int ctas) {
  if (dev < 0 || dev >= 64) return;
  g_tuned_ctas[dev][l_bucket(l)] = std::max(0, ctas);
}

int tuned_jacobi_threads(int dev, int l) {
  if (dev < 0 || dev >= 64) return 0;
  return g_tuned_threads[dev][l_bucket(l)];
}

void set_tuned_jacobi_threads(int dev, int l, int threads) {
  if (dev < 0 || dev >= 64) return;
  g_tuned_threads[dev][l_bucket(l)] = (threads == 256 || threads == 512 || threads == 1024) ? threads : 0;
}

namespace {
// The cooperative kernel's instantiation for NT threads per CTA and its CTAs per SM.
const void* coop_kernel(int nt) {
  if (nt == 256) return (const void*)k_jacobi_coop<double, 256>;
  if (nt == 1024) return (const void*)k_jacobi_coop<double, 1024>;
  return (const void*)k_jacobi_coop<double, 512>;
}
}  // namespace

int jacobi_sym_f64(cudaStream_t st, int l, const double* Z, const double* warm, double* P,
                   double* sig, JacobiWork& w, int max_sweeps, double* host_scal, int ctas) {
  const int lp = std::max(2, l + (l & 1));   // even, >= 2; a zero pad row/column never rotates
  const int half = lp / 2;
  int dev = 0, nsm = 0, per_sm = 0;
  KOT_CUDA(cudaGetDevice(&dev));
  KOT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  // threads per CTA: the caller's probe, else the autotuner's choice for this size bucket, else 512
  int nt = w.threads_override > 0 ? w.threads_override : tuned_jacobi_threads(dev, l);
  if (nt != 256 && nt != 1024) nt = kCoopThreads;
  KOT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, coop_kernel(nt), nt, 0));
  if (per_sm < 1) throw Error{KOT_ERR_CUDA, "eig: cooperative kernel does not fit on an SM"};
  // one CTA per SM by default (fewer arrivals per barrier than several per SM), or the
  // autotuner's choice for this size bucket
  if (ctas <= 0) ctas = tuned_jacobi_ctas(dev, l);
  const int grid = ctas > 0 ? std::min(ctas, nsm * per_sm) : nsm;
  w.A.alloc(2 * (size_t)lp * lp);
  w.V.alloc((size_t)lp * lp);
  w.rot.alloc(2 * (size_t)lp);
  w.rank.alloc((size_t)l);
  w.partial.alloc(std::max<size_t>(kReduceBlocks, 2 * (size_t)grid));
  w.scal.alloc(4);
  w.bar.alloc(2);
  KOT_CUDA(cudaMemsetAsync(w.bar.p, 0, 2 * sizeof(unsigned), st));   // counters start at 0
  w.flags.alloc(2);
  KOT_CUDA(cudaMemsetAsync(w.flags.p, 0, 2 * sizeof(int), st));
  double* A0 = w.A.p;
  double* A1 = w.A.p + (size_t)lp * lp;
  dim3 g2(cdiv(lp, 32), cdiv(lp, 8)), b2(32, 8);
  if (warm) {
    // A = warm^T Z warm: V(:, :l) = Z warm (ld lp), then A0 = warm^T V
    gemm_acc(st, w.oz, false, false, l, l, l, 1.0, Z, l, warm, l, nullptr, 0.0, w.V.p, lp, 0);
    gemm_acc(st, w.oz, true, false, l, l, l, 1.0, warm, l, w.V.p, lp, nullptr, 0.0, A0, lp, G_SYM);
    k_init_pad<<<g2, b2, 0, st>>>(l, lp, A0, w.V.p, nullptr, warm);
  } else {
    k_init_pad<<<g2, b2, 0, st>>>(l, lp, A0, w.V.p, Z, nullptr);
  }
  KOT_CHECK_LAUNCH();
  CoopArgs<double> a;
  a.lp = lp;
  a.l = l;
  a.max_sweeps = max_sweeps;
  a.A0 = A0;
  a.A1 = A1;
  a.V = w.V.p;
  a.rot0 = w.rot.p;
  a.rot1 = w.rot.p + lp;
  a.partial = w.partial.p;
  a.bar = w.bar.p;
  a.err = w.flags.p;
  a.sweeps_out = w.flags.p + 1;
  a.tol_rel = 1e-14;
  a.floor_rel = 1e-12;
  {
    // algorithmic work of one sweep: (lp - 1) rounds of 24 flops per 2x2 block of A over the
    // upper half of the (lp/2)^2 blocks and 6 flops per (row, pair) of V
    const double hb = (double)half * (half + 1) / 2.0;
    const double rflops = 24.0 * hb + 6.0 * (double)l * half;
    ProfScope ps(st, KC_JACOBI, rflops * (lp - 1), 8.0 * 2.0 * (2.0 * lp * (double)lp + (double)l * lp));
    void* args[] = {&a};
    KOT_CUDA(cudaLaunchCooperativeKernel(coop_kernel(nt), dim3(grid), dim3(nt), args, 0, st));
    KOT_LAUNCHED(1);
  }
  int hflags[2] = {0, 0};
  KOT_CUDA(cudaMemcpyAsync(hflags, w.flags.p, sizeof(hflags), cudaMemcpyDeviceToHost, st));
  KOT_CUDA(cudaStreamSynchronize(st));
  (void)host_scal;
  if (hflags[0] == 1) throw Error{KOT_ERR_TIMEOUT, "eig: grid barrier timed out"};
  if (hflags[0] == 2) throw Error{KOT_ERR_NO_CONVERGENCE, "eig: Jacobi did not converge"};
  const int sweeps = hflags[1] / 2, cur = hflags[1] & 1;
  const double* Af = cur ? A1 : A0;
  k_rank_stride<<<cdiv(l, 32), dim3(32, 8), 0, st>>>(l, Af, lp + 1, w.rank.p);
  k_gather<<<dim3(cdiv(l, 32), cdiv(l, 8)), b2, 0, st>>>(l, lp, Af, w.V.p, w.rank.p, P, sig);
  KOT_LAUNCHED(2);
  return sweeps;
}

}  // namespace kot
