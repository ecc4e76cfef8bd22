// Dense FP64 building blocks: tiled GEMM with triangular k-range cuts, GEMV, deterministic
// reductions and elementwise helpers.
//
// FP64 on GB300 issues about two fused multiply-adds per clock per SM, so these kernels are
// bound by the FP64 pipe: the design goal is to keep all 152 SMs busy (small 32 x 32 tiles) and
// to skip work the triangular Cholesky factor makes zero, not to stage operands for tensor cores.
#include <algorithm>
#include <cstdlib>
#include <atomic>
#include <map>
#include <mutex>
#include <utility>

#include "kot_internal.cuh"

namespace kot {

static std::atomic<long long> g_launches{0};
void note_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long launch_total() { return g_launches.load(std::memory_order_relaxed); }

static thread_local Profiler* t_prof = nullptr;
Profiler* current_profiler() { return t_prof; }
void set_current_profiler(Profiler* p) { t_prof = p; }

cudaEvent_t Profiler::get_event() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  KOT_CUDA(cudaEventCreate(&e));
  return e;
}

void Profiler::begin(cudaStream_t st, int cls, cudaEvent_t* a) {
  std::lock_guard<std::mutex> lk(mu);
  *a = get_event();
  KOT_CUDA(cudaEventRecord(*a, st));
}

void Profiler::end(cudaStream_t st, int cls, cudaEvent_t a, double fl, double by, double ex) {
  std::lock_guard<std::mutex> lk(mu);
  cudaEvent_t b = get_event();
  if (cudaEventRecord(b, st) != cudaSuccess) return;
  pending.push_back({cls, a, b, fl, by, ex});
  if (pending.size() > 4096) collect_locked();
}

void Profiler::collect() {
  std::lock_guard<std::mutex> lk(mu);
  collect_locked();
}

void Profiler::collect_locked() {
  for (auto& q : pending) {
    float t = 0.f;
    if (cudaEventSynchronize(q.b) == cudaSuccess && cudaEventElapsedTime(&t, q.a, q.b) == cudaSuccess) {
      launches[q.cls] += 1;
      ms[q.cls] += t;
      flops[q.cls] += q.flops;
      bytes[q.cls] += q.bytes;
      exec[q.cls] += q.exec;
    }
    pool.push_back(q.a);
    pool.push_back(q.b);
  }
  pending.clear();
}

void Profiler::reset() {
  std::lock_guard<std::mutex> lk(mu);
  collect_locked();
  for (int i = 0; i < KC_COUNT; ++i) launches[i] = seen[i] = 0, ms[i] = flops[i] = bytes[i] = exec[i] = 0.0;
}

void Profiler::release() {
  std::lock_guard<std::mutex> lk(mu);
  collect_locked();
  for (auto e : pool) cudaEventDestroy(e);
  pool.clear();
}

namespace {

// ------------------------------------------------------------------ FP64 GEMM (stream-K)
// C = alpha op(A) diag(s) op(B) + beta C on the FP64 pipes.  FP64 issue is the bound (two FMA
// per clock per SM on this part), so the design goal is that every SM sub-partition gets the
// same number of FMAs: the grid is one CTA of eight warps per SM,
// the output is cut into 16 x 16 warp tiles, the (tile, k) iterations of all tiles are laid
// end to end and every warp takes an equal contiguous share ("stream-K").  Two warps share each
// sub-partition so that one issues while the other waits on memory.  A tile finished by
// one warp is stored directly; a tile shared by several warps is summed from their partials in
// warp order by whichever of them arrives last (per-tile arrival counter), so the result does
// not depend on timing.  Operands are staged per warp through shared memory in k-chunks of 16,
// the next chunk held in registers while the current one is multiplied.
constexpr int SK_T = 16, SK_KC = 16, SK_WARPS = 8;
constexpr int SK_P = SK_T + 2;   // row pitch of the staged tiles (16-byte aligned rows)

struct SkArgs {
  int M, N, K, flags;
  double alpha, beta;
  const double* A;
  const double* B;
  const double* s;
  double* C;
  int lda, ldb, ldc;
  int tn;              // tile columns
  int ntiles;          // tiles in the work list (upper triangle only for G_SYM)
  int W;               // warps taking part
  long long T;         // iterations over all tiles
  double* part;        // W x 2 x 256 partial tiles
  unsigned* cnt;       // ntiles arrival counters (zero between launches)
};

// Tile t of the work list: origin (m0, n0), k-range [kb, ke) and its length in the iteration
// space (at least 1, so that a tile with an empty k-range still gets written).
__host__ __device__ inline void sk_tile(int flags, int K, int tn, int t, int& m0, int& n0, int& kb,
                                        int& ke, int& len) {
  int ti, tj;
  if (flags & G_SYM) {
    // upper triangle row by row: row i starts at i*tn - i*(i-1)/2
    const float b = 2.0f * tn + 1.0f;
    ti = (int)((b - sqrtf(fmaxf(b * b - 8.0f * t, 0.0f))) * 0.5f);   // estimate, fixed below
    if (ti < 0) ti = 0;
    while (ti > 0 && (long long)ti * tn - (long long)ti * (ti - 1) / 2 > t) --ti;
    while ((long long)(ti + 1) * tn - (long long)(ti + 1) * ti / 2 <= t) ++ti;
    tj = ti + (int)(t - ((long long)ti * tn - (long long)ti * (ti - 1) / 2));
  } else {
    ti = t / tn;
    tj = t - ti * tn;
  }
  m0 = ti * SK_T;
  n0 = tj * SK_T;
  kb = 0;
  ke = K;
  if (flags & G_KLO_ROW) kb = kb > m0 ? kb : m0;
  if (flags & G_KLO_COL) kb = kb > n0 ? kb : n0;
  if (flags & G_KHI_COL) ke = ke < n0 + SK_T ? ke : n0 + SK_T;
  if (flags & G_KHI_ROW) ke = ke < m0 + SK_T ? ke : m0 + SK_T;
  len = ke - kb > 1 ? ke - kb : 1;
}

// warp holding iteration g (shares floor(w T / W))
__device__ __forceinline__ int sk_owner(long long g, long long T, int W) {
  return (int)(((g + 1) * (long long)W - 1) / T);
}

// Chunk of 16 k: each operand tile is 16 x 16, eight values per lane, read as rows of 16
// consecutive doubles (two rows per warp instruction).
template <bool TA, bool TB>
__device__ __forceinline__ void sk_load(const SkArgs& a, int m0, int n0, int kc, int kz, int lane,
                                        double (&ra)[8], double (&rb)[8]) {
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    int m, k;
    if (TA) { k = kc + 2 * q + (lane >> 4); m = m0 + (lane & 15); }
    else { k = kc + (lane & 15); m = m0 + 2 * q + (lane >> 4); }
    double v = 0.0;
    if (m < a.M && k < kz) {
      v = TA ? a.A[(size_t)k * a.lda + m] : a.A[(size_t)m * a.lda + k];
      if (a.s) v *= a.s[k];
    }
    ra[q] = v;
    int n, kk;
    if (TB) { kk = kc + (lane & 15); n = n0 + 2 * q + (lane >> 4); }
    else { kk = kc + 2 * q + (lane >> 4); n = n0 + (lane & 15); }
    double w = 0.0;
    if (n < a.N && kk < kz) w = TB ? a.B[(size_t)n * a.ldb + kk] : a.B[(size_t)kk * a.ldb + n];
    rb[q] = w;
  }
}

template <bool TA, bool TB>
__device__ __forceinline__ void sk_stage(int lane, const double (&ra)[8], const double (&rb)[8],
                                         double (*sA)[SK_P], double (*sB)[SK_P]) {
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    if (TA) sA[2 * q + (lane >> 4)][lane & 15] = ra[q];
    else sA[lane & 15][2 * q + (lane >> 4)] = ra[q];
    if (TB) sB[lane & 15][2 * q + (lane >> 4)] = rb[q];
    else sB[2 * q + (lane >> 4)][lane & 15] = rb[q];
  }
}

// G_SYM: only entries on or above the diagonal are stored, each also at its mirror position, so
// the result is exactly symmetric.  (A diagonal tile holds both (m, n) and (n, m); storing both
// as computed would leave their rounding-level difference in C, and a symmetric matrix that is
// not exactly so lets that antisymmetric part grow through the 1/mu weights of T_k, Sec. 4.3.)
__device__ __forceinline__ void sk_store(const SkArgs& a, int m0, int n0, int r, int c,
                                         const double (&acc)[2][4]) {
  const bool sym = (a.flags & G_SYM) != 0;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int gm = m0 + 2 * r + i;
    if (gm >= a.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + 4 * c + j;
      if (gn >= a.N || (sym && gn < gm)) continue;
      const bool mirror = sym && gn > gm;
      const double v = a.alpha * acc[i][j];
      double* cp = &a.C[(size_t)gm * a.ldc + gn];
      *cp = (a.beta == 0.0) ? v : v + a.beta * (*cp);
      if (mirror) {
        double* cm = &a.C[(size_t)gn * a.ldc + gm];
        *cm = (a.beta == 0.0) ? v : v + a.beta * (*cm);
      }
    }
  }
}

template <bool TA, bool TB>
__global__ void __launch_bounds__(32 * SK_WARPS, 1) k_gemm_f64_sk(SkArgs a) {
  __shared__ __align__(16) double sA[SK_WARPS][SK_KC][SK_P];
  __shared__ __align__(16) double sB[SK_WARPS][SK_KC][SK_P];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int w = wl * gridDim.x + blockIdx.x;   // consecutive shares on different SMs
  if (w >= a.W) return;
  const long long g0 = (long long)w * a.T / a.W, g1 = (long long)(w + 1) * a.T / a.W;
  if (g0 >= g1) return;
  // locate the tile holding g0: scan the tile lengths 32 at a time
  int t = 0;
  long long st = 0;
  for (int tb = 0; tb < a.ntiles; tb += 32) {
    int len = 0;
    if (tb + lane < a.ntiles) {
      int m0, n0, kb, ke;
      sk_tile(a.flags, a.K, a.tn, tb + lane, m0, n0, kb, ke, len);
    }
    long long incl = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    const long long tot = __shfl_sync(0xffffffffu, incl, 31);
    if (g0 < st + tot) {
      const unsigned mask = __ballot_sync(0xffffffffu, st + incl > g0);
      const int L = __ffs(mask) - 1;
      const long long incl_L = __shfl_sync(0xffffffffu, incl, L);
      const int len_L = __shfl_sync(0xffffffffu, len, L);
      t = tb + L;
      st += incl_L - len_L;
      break;
    }
    st += tot;
  }
  const int r = lane >> 2, c = lane & 3;
  double (*wA)[SK_P] = sA[wl];
  double (*wB)[SK_P] = sB[wl];
  long long g = g0;
  while (g < g1) {
    int m0, n0, kb, ke, len;
    sk_tile(a.flags, a.K, a.tn, t, m0, n0, kb, ke, len);
    const long long et = st + len, pe = et < g1 ? et : g1;
    const int ka = kb + (int)(g - st);
    const int kz = min(ke, kb + (int)(pe - st));
    double acc[2][4] = {{0.0, 0.0, 0.0, 0.0}, {0.0, 0.0, 0.0, 0.0}};
    if (ka < kz) {
      double ra[8], rb[8];
      sk_load<TA, TB>(a, m0, n0, ka, kz, lane, ra, rb);
      for (int kc = ka; kc < kz; kc += SK_KC) {
        __syncwarp();
        sk_stage<TA, TB>(lane, ra, rb, wA, wB);
        __syncwarp();
        if (kc + SK_KC < kz) sk_load<TA, TB>(a, m0, n0, kc + SK_KC, kz, lane, ra, rb);
        const int nk = min(SK_KC, kz - kc);
#pragma unroll 4
        for (int k = 0; k < nk; ++k) {
          const double2 av = *reinterpret_cast<const double2*>(&wA[k][2 * r]);
          const double2 b01 = *reinterpret_cast<const double2*>(&wB[k][4 * c]);
          const double2 b23 = *reinterpret_cast<const double2*>(&wB[k][4 * c + 2]);
          const double b[4] = {b01.x, b01.y, b23.x, b23.y};
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            acc[0][j] = fma(av.x, b[j], acc[0][j]);
            acc[1][j] = fma(av.y, b[j], acc[1][j]);
          }
        }
      }
    }
    if (g == st && pe == et) {
      sk_store(a, m0, n0, r, c, acc);
    } else {
      // partial tile: slot 0 for the warp's first piece, slot 1 for its last
      const int slot = (g == g0) ? 0 : 1;
      double* mine = a.part + ((size_t)w * 2 + slot) * 256 + lane * 8;
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mine[i * 4 + j] = acc[i][j];
      __threadfence();
      __syncwarp();
      const int wa = sk_owner(st, a.T, a.W), wb = sk_owner(et - 1, a.T, a.W);
      unsigned old = 0;
      if (lane == 0) old = atomicAdd(&a.cnt[t], 1u);
      old = __shfl_sync(0xffffffffu, old, 0);
      if (old == (unsigned)(wb - wa)) {
        __threadfence();
        double sum[2][4] = {{0.0, 0.0, 0.0, 0.0}, {0.0, 0.0, 0.0, 0.0}};
        for (int v = wa; v <= wb; ++v) {
          const long long gv = (long long)v * a.T / a.W;
          const int sv = (v == wa && gv < st) ? 1 : 0;
          const double* src = a.part + ((size_t)v * 2 + sv) * 256 + lane * 8;
#pragma unroll
          for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) sum[i][j] += __ldcg(src + i * 4 + j);
        }
        sk_store(a, m0, n0, r, c, sum);
        if (lane == 0) a.cnt[t] = 0u;   // ready for the next launch on this stream
      }
    }
    g = pe;
    st = et;
    ++t;
  }
}

// out[i] = sum_{a <= i} R[a,i] Y[a,i]: 32 columns per block, 32 rows of threads striding a
// (coalesced across i), partial sums reduced through shared memory.
__global__ void __launch_bounds__(1024) k_coldot_upper(int l, const double* __restrict__ R,
                                                       const double* __restrict__ Y, double* __restrict__ out) {
  pdl_wait();
  pdl_trigger();
  __shared__ double part[32][33];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i = blockIdx.x * 32 + tx;
  double acc0 = 0.0, acc1 = 0.0;
  if (i < l) {
    int a = ty;
    for (; a + 32 <= i; a += 64) {
      acc0 = fma(R[(size_t)a * l + i], Y[(size_t)a * l + i], acc0);
      acc1 = fma(R[(size_t)(a + 32) * l + i], Y[(size_t)(a + 32) * l + i], acc1);
    }
    if (a <= i) acc0 = fma(R[(size_t)a * l + i], Y[(size_t)a * l + i], acc0);
  }
  part[ty][tx] = acc0 + acc1;
  __syncthreads();
  if (ty == 0 && i < l) {
    double s = 0.0;
#pragma unroll 8
    for (int r = 0; r < 32; ++r) s += part[r][tx];
    out[i] = s;
  }
}

// One 32 x 32 block per 32 columns: lane tx owns column i, row group ty strides the rows.
__global__ void __launch_bounds__(1024) k_coldot_rows(int rows, int n, const double* __restrict__ A, int lda,
                                                      const double* __restrict__ Y, int ldy, double scale,
                                                      double* __restrict__ out) {
  pdl_wait();
  pdl_trigger();
  __shared__ double part[32][33];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i = blockIdx.x * 32 + tx;
  double acc0 = 0.0, acc1 = 0.0;
  if (i < n) {
    int a = ty;
    for (; a + 32 < rows; a += 64) {
      acc0 = fma(A[(size_t)a * lda + i], Y[(size_t)a * ldy + i], acc0);
      acc1 = fma(A[(size_t)(a + 32) * lda + i], Y[(size_t)(a + 32) * ldy + i], acc1);
    }
    if (a < rows) acc0 = fma(A[(size_t)a * lda + i], Y[(size_t)a * ldy + i], acc0);
  }
  part[ty][tx] = acc0 + acc1;
  __syncthreads();
  if (ty == 0 && i < n) {
    double s = 0.0;
#pragma unroll 8
    for (int r = 0; r < 32; ++r) s += part[r][tx];
    out[i] = scale * s;
  }
}

__global__ void k_gemv(int n, double alpha, const double* __restrict__ A,
                       const double* __restrict__ x, double beta, double* __restrict__ y) {
  pdl_wait();
  pdl_trigger();
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n) return;
  const double* row = A + (size_t)warp * n;
  double acc = 0.0;
  for (int j = lane; j < n; j += 32) acc = fma(row[j], x[j], acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) y[warp] = alpha * acc + (beta == 0.0 ? 0.0 : beta * y[warp]);
}

template <int NT>
__device__ double block_sum(double v, double* sh) {
  const int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
#pragma unroll
  for (int o = NT / 2; o > 0; o >>= 1) {
    if (t < o) sh[t] += sh[t + o];
    __syncthreads();
  }
  return sh[0];
}

__global__ void k_dot_partial(size_t n, const double* __restrict__ x, const double* __restrict__ y,
                              double* __restrict__ partial) {
  pdl_wait();
  pdl_trigger();
  __shared__ double sh[256];
  double acc = 0.0;
  for (size_t i = blockIdx.x * 256 + threadIdx.x; i < n; i += (size_t)gridDim.x * 256)
    acc = fma(x[i], y ? y[i] : x[i], acc);
  double s = block_sum<256>(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void k_sum_partials(int nb, const double* __restrict__ partial, double* __restrict__ out) {
  pdl_wait();
  pdl_trigger();
  __shared__ double sh[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nb; i += 256) acc += partial[i];
  double s = block_sum<256>(acc, sh);
  if (threadIdx.x == 0) *out = s;
}

// Single-block reduction for short arrays (one launch instead of partials + sum):
// *out = sum_i x_i y_i (y null: sum x_i^2), fixed summation order.
__global__ void __launch_bounds__(1024) k_dot_one(size_t n, const double* __restrict__ x,
                                                  const double* __restrict__ y, double* __restrict__ out) {
  pdl_wait();
  pdl_trigger();
  __shared__ double sh[1024];
  double acc = 0.0;
  for (size_t i = threadIdx.x; i < n; i += 1024) acc = fma(x[i], y ? y[i] : x[i], acc);
  const double s = block_sum<1024>(acc, sh);
  if (threadIdx.x == 0) *out = s;
}

// One CG step on the device (single block; n is the length of the vectors): with ee = sc[5+cur],
//   pHp = p.Hp -> sc[3];  a = ee / pHp;  x += a p;  e -= a Hp;  ee' = |e|^2 -> sc[5+(cur^1)];
//   p = e + (ee'/ee) p.
// pHp <= 0: nothing is updated, sc[7] = 1 and sc[5+(cur^1)] = ee.
// W (nw entries, may be null) += a Wp: a quantity carried along x, e.g. the rows of T[Phi*(x)].
__global__ void __launch_bounds__(1024) k_cg_step(int n, const double* __restrict__ Hp, double* __restrict__ p,
                                                  double* __restrict__ x, double* __restrict__ e,
                                                  double* __restrict__ sc, int cur, size_t nw,
                                                  const double* __restrict__ Wp, double* __restrict__ W) {
  pdl_wait();
  pdl_trigger();
  __shared__ double sh[1024];
  const int t = threadIdx.x;
  double acc = 0.0;
  for (int i = t; i < n; i += 1024) acc = fma(p[i], Hp[i], acc);
  const double pHp = block_sum<1024>(acc, sh);
  const double ee = sc[5 + cur];
  __syncthreads();
  if (t == 0) sc[3] = pHp;
  if (!(pHp > 0.0)) {
    if (t == 0) {
      sc[7] = 1.0;
      sc[5 + (cur ^ 1)] = ee;
    }
    return;
  }
  const double a = ee / pHp;
  if (W)
    for (size_t i = t; i < nw; i += 1024) W[i] = fma(a, Wp[i], W[i]);
  acc = 0.0;
  for (int i = t; i < n; i += 1024) {
    x[i] = fma(a, p[i], x[i]);
    const double ei = fma(-a, Hp[i], e[i]);
    e[i] = ei;
    acc = fma(ei, ei, acc);
  }
  const double ee1 = block_sum<1024>(acc, sh);
  if (t == 0) sc[5 + (cur ^ 1)] = ee1;
  const double b = ee1 / ee;
  for (int i = t; i < n; i += 1024) p[i] = fma(b, p[i], e[i]);
}

// Norms of the inexact-Newton test: out[0] = |x|^2 (n1 entries), out[1] = |a - b|^2 (n2 entries).
// One block writes out directly; several blocks write partial pairs that k_sum_pairs adds.
__global__ void k_two_norms(size_t n1, const double* __restrict__ x, size_t n2, const double* __restrict__ a,
                            const double* __restrict__ b, double* __restrict__ out) {
  pdl_wait();
  pdl_trigger();
  __shared__ double sh[256];
  double s1 = 0.0, s2 = 0.0;
  const size_t stride = (size_t)gridDim.x * 256;
  for (size_t i = blockIdx.x * 256 + threadIdx.x; i < n1; i += stride) s1 = fma(x[i], x[i], s1);
  for (size_t i = blockIdx.x * 256 + threadIdx.x; i < n2; i += stride) {
    const double d = a[i] - b[i];
    s2 = fma(d, d, s2);
  }
  s1 = block_sum<256>(s1, sh);
  __syncthreads();
  s2 = block_sum<256>(s2, sh);
  if (threadIdx.x == 0) {
    out[2 * blockIdx.x] = s1;
    out[2 * blockIdx.x + 1] = s2;
  }
}

__global__ void k_eig_norms(size_t n1, const double* __restrict__ x, int rows, int cols, int ld, int nb,
                            const double* __restrict__ A, const double* __restrict__ W,
                            const double* __restrict__ base, double* __restrict__ out) {
  pdl_wait();
  pdl_trigger();
  __shared__ double sh[256];
  double s1 = 0.0, s2 = 0.0;
  const size_t stride = (size_t)gridDim.x * 256;
  for (size_t i = blockIdx.x * 256 + threadIdx.x; i < n1; i += stride) s1 = fma(x[i], x[i], s1);
  const size_t n2 = (size_t)rows * cols;
  for (size_t i = blockIdx.x * 256 + threadIdx.x; i < n2; i += stride) {
    const int r = (int)(i / cols), j = (int)(i - (size_t)r * cols);
    const size_t o = (size_t)r * ld + j;
    const bool bar = j < nb;
    const double d = A[o] - (W ? (bar ? 1.0 : 2.0) * W[o] : 0.0);
    s2 = fma(bar ? 2.0 * d : d, d, s2);
  }
  if (base && blockIdx.x == 0 && threadIdx.x == 0) s2 += *base;
  s1 = block_sum<256>(s1, sh);
  __syncthreads();
  s2 = block_sum<256>(s2, sh);
  if (threadIdx.x == 0) {
    out[2 * blockIdx.x] = s1;
    out[2 * blockIdx.x + 1] = s2;
  }
}

__global__ void k_sum_pairs(int nb, const double* __restrict__ partial, double* __restrict__ out) {
  pdl_wait();
  pdl_trigger();
  __shared__ double sh[256];
  double s1 = 0.0, s2 = 0.0;
  for (int i = threadIdx.x; i < nb; i += 256) {
    s1 += partial[2 * i];
    s2 += partial[2 * i + 1];
  }
  s1 = block_sum<256>(s1, sh);
  __syncthreads();
  s2 = block_sum<256>(s2, sh);
  if (threadIdx.x == 0) {
    out[0] = s1;
    out[1] = s2;
  }
}

// y = alpha A x + mu x + v  (A: n x n row-major; v may be null)
__global__ void k_hmatvec(int n, double alpha, const double* __restrict__ A, const double* __restrict__ x,
                          double mu, const double* __restrict__ v, double* __restrict__ y) {
  pdl_wait();
  pdl_trigger();
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n) return;
  const double* row = A + (size_t)warp * n;
  double acc = 0.0;
  for (int j = lane; j < n; j += 32) acc = fma(row[j], x[j], acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) {
    double r = fma(mu, x[warp], alpha * acc);
    if (v) r += v[warp];
    y[warp] = r;
  }
}

__global__ void k_axpby(size_t n, double a, const double* __restrict__ x, double b,
                        const double* __restrict__ y, double* __restrict__ out) {
  pdl_wait();
  pdl_trigger();
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    double v = a * x[i];
    if (y) v = fma(b, y[i], v);
    out[i] = v;
  }
}

// y += sgn * (num / den) x with the ratio read from device memory; den <= 0 (or NaN) leaves y
// unchanged and sets *flag = 1 (block 0 writes it) when flag is given.
__global__ void k_axpy_ratio(size_t n, const double* __restrict__ num, const double* __restrict__ den,
                             double sgn, const double* __restrict__ x, double* __restrict__ y,
                             double* __restrict__ flag) {
  pdl_wait();
  pdl_trigger();
  const double dn = *den;
  if (!(dn > 0.0)) {
    if (flag && blockIdx.x == 0 && threadIdx.x == 0) *flag = 1.0;
    return;
  }
  const double a = sgn * (*num / dn);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = fma(a, x[i], y[i]);
}

// y = x + (num / den) y with the ratio read from device memory
__global__ void k_xpby_ratio(size_t n, const double* __restrict__ x, const double* __restrict__ num,
                             const double* __restrict__ den, double* __restrict__ y) {
  pdl_wait();
  pdl_trigger();
  const double b = *num / *den;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = fma(b, y[i], x[i]);
}

// Z = sym(X - a S) - c I (the argument of the projection in Eq. 4.2 and in the EG steps; S null
// reads as zero) and, if FX is given, FX = S + c I (the X part of the EG operator at the same
// point, with a = 1); one thread per pair i <= j.
__global__ void k_form_z(int l, const double* __restrict__ X, const double* __restrict__ S, double a, double c,
                         double* __restrict__ Z, double* __restrict__ FX) {
  pdl_wait();
  pdl_trigger();
  const int j = blockIdx.x * 32 + threadIdx.x, i = blockIdx.y * 8 + threadIdx.y;
  if (i >= l || j >= l || j < i) return;
  const size_t ij = (size_t)i * l + j, ji = (size_t)j * l + i;
  if (i == j) {
    const double sii = S ? S[ij] : 0.0;
    Z[ij] = (X[ij] - a * sii) - c;
    if (FX) FX[ij] = sii + c;
    return;
  }
  const double sij = S ? S[ij] : 0.0, sji = S ? S[ji] : 0.0;
  const double v = 0.5 * ((X[ij] - a * sij) + (X[ji] - a * sji));
  Z[ij] = v;
  Z[ji] = v;
  if (FX) {
    FX[ij] = sij;
    FX[ji] = sji;
  }
}

// out_i = s (Q gamma)_i - s z_i - v_i (one warp per row): the gradient of Eq. 4.1's Lagrangian in
// gamma, i.e. r1 of Eq. 4.2, with v = Phi(X).
__global__ void k_grad_gamma(int n, double s, const double* __restrict__ Q, const double* __restrict__ gamma,
                             const double* __restrict__ z, const double* __restrict__ v,
                             double* __restrict__ out) {
  pdl_wait();
  pdl_trigger();
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n) return;
  const double* row = Q + (size_t)warp * n;
  double acc = 0.0;
  for (int j = lane; j < n; j += 32) acc = fma(row[j], gamma[j], acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) out[warp] = (s * acc - s * z[warp]) - v[warp];
}

// D = X - P (elementwise over n2 entries) with partial sums of |x1|^2 (n1 entries) and |D|^2:
// the residual block r2 of Eq. 4.2 and both norms of ||R(w)||; pairs as in k_two_norms.
__global__ void k_sub_norms(size_t n1, const double* __restrict__ x1, size_t n2, const double* __restrict__ X,
                            const double* __restrict__ P, double* __restrict__ D, double* __restrict__ out) {
  pdl_wait();
  pdl_trigger();
  __shared__ double sh[256];
  double s1 = 0.0, s2 = 0.0;
  const size_t stride = (size_t)gridDim.x * 256;
  for (size_t i = blockIdx.x * 256 + threadIdx.x; i < n1; i += stride) s1 = fma(x1[i], x1[i], s1);
  for (size_t i = blockIdx.x * 256 + threadIdx.x; i < n2; i += stride) {
    const double d = X[i] - P[i];
    D[i] = d;
    s2 = fma(d, d, s2);
  }
  s1 = block_sum<256>(s1, sh);
  __syncthreads();
  s2 = block_sum<256>(s2, sh);
  if (threadIdx.x == 0) {
    out[2 * blockIdx.x] = s1;
    out[2 * blockIdx.x + 1] = s2;
  }
}

__global__ void k_square(size_t n, const double* __restrict__ x, double* __restrict__ out) {
  pdl_wait();
  pdl_trigger();
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    out[i] = x[i] * x[i];
}

__global__ void k_fill(size_t n, double v, double* __restrict__ out) {
  pdl_wait();
  pdl_trigger();
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    out[i] = v;
}

__global__ void k_symmetrize(int l, double* A) {
  pdl_wait();
  pdl_trigger();
  const int j = blockIdx.x * 32 + threadIdx.x, i = blockIdx.y * 8 + threadIdx.y;
  if (i < l && j < l && i < j) {
    double v = 0.5 * (A[(size_t)i * l + j] + A[(size_t)j * l + i]);
    A[(size_t)i * l + j] = v;
    A[(size_t)j * l + i] = v;
  }
}

__global__ void k_add_diag(int l, double v, double* A, int lda) {
  pdl_wait();
  pdl_trigger();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < l) A[(size_t)i * lda + i] += v;
}

__global__ void k_copy_mat(int rows, int cols, const double* __restrict__ A, int lda,
                           double* __restrict__ B, int ldb) {
  pdl_wait();
  pdl_trigger();
  const int j = blockIdx.x * 32 + threadIdx.x, i = blockIdx.y * 8 + threadIdx.y;
  if (i < rows && j < cols) B[(size_t)i * ldb + j] = A[(size_t)i * lda + j];
}

__global__ void k_sym_sum(int l, const double* __restrict__ G, const double* __restrict__ S,
                          double inv_mu, int complement, double* __restrict__ out) {
  pdl_wait();
  pdl_trigger();
  const int j = blockIdx.x * 32 + threadIdx.x, i = blockIdx.y * 8 + threadIdx.y;
  if (i >= l || j >= l) return;
  double g = G[(size_t)i * l + j] + G[(size_t)j * l + i];
  out[(size_t)i * l + j] = complement ? fma(inv_mu, S[(size_t)i * l + j], -g) : g;
}

inline int cdiv(size_t a, int b) { return (int)((a + b - 1) / b); }
// grid of the elementwise helpers: at least one block, so that n = 0 is a valid (empty) launch
inline int elementwise_grid(size_t n) { return std::max(1, std::min(cdiv(n, 256), 1216)); }

}  // namespace

bool pdl_enabled() {
  static const bool on = [] {
    const char* v = std::getenv("KOT_PDL");
    return !(v && v[0] == '0' && v[1] == '\0');
  }();
  return on;
}

namespace {

// Per-stream scratch of the stream-K GEMM (partials and arrival counters).  Launches on one
// stream are ordered, so one set per stream suffices; counters are left at zero by every launch.
struct SkWork {
  DevBuf<double> part;
  DevBuf<unsigned> cnt;
};
std::mutex g_sk_mu;
std::map<std::pair<int, cudaStream_t>, SkWork> g_sk;

// Multiply-adds the product needs (what the kernel computes, excluding skipped zero blocks):
// rows m, columns n >= m under G_SYM, and k in [max(lo_row, lo_col), min(hi_row, hi_col)).
double gemm_macs(int M, int N, int K, int flags) {
  const bool sym = flags & G_SYM, klc = flags & G_KLO_COL, khc = flags & G_KHI_COL;
  double macs = 0.0;
  for (long m = 0; m < M; ++m) {
    const long a = (flags & G_KLO_ROW) ? m : 0;
    const long b = (flags & G_KHI_ROW) ? std::min<long>(m + 1, K) : K;
    const long n0 = sym ? m : 0, n1 = N;
    if (n0 >= n1 || b <= a) continue;
    if (!klc && !khc) {
      macs += (double)(n1 - n0) * (b - a);
    } else if (klc && !khc) {   // count(n) = b - max(a, n)
      const long lo = std::max(n0, a), hi = std::min(n1, b);
      macs += (double)std::max(0L, std::min(n1, a) - n0) * (b - a);
      if (hi > lo) macs += (double)(hi - lo) * (2 * b - lo - hi + 1) / 2.0;
    } else if (!klc && khc) {   // count(n) = min(b, n + 1) - a
      const long lo = std::max(n0, a), hi = std::min(n1, b);
      if (hi > lo) macs += (double)(hi - lo) * (lo + hi + 1 - 2 * a) / 2.0;
      macs += (double)std::max(0L, n1 - std::max(n0, b)) * (b - a);
    } else {
      for (long n = n0; n < n1; ++n) macs += (double)std::max(0L, std::min(b, n + 1) - std::max(a, n));
    }
  }
  return macs;
}

// Short inner dimension (K <= kLowK, e.g. the l x l x min(|alpha|, |alpha-bar|) product of the
// projection, Eq. (4.4)): C = alpha A diag(s) B^T + beta C with A (M x K) and B (N x K) row-major.
// One 32 x 32 tile of C per block with both K-wide panels staged whole in shared memory, so the
// kernel is one pass over C; the stream-K GEMM spends most of its time on set-up at such K.
// G_SYM: blocks enumerate the tiles on or above the diagonal and store like sk_store.
constexpr int kLowK = 64;
__global__ void __launch_bounds__(256) k_gemm_f64_lowk(int M, int N, int K, double alpha,
                                                       const double* __restrict__ A, int lda,
                                                       const double* __restrict__ B, int ldb,
                                                       const double* __restrict__ s, double beta,
                                                       double* C, int ldc, int sym, int tn) {
  pdl_wait();
  pdl_trigger();
  __shared__ double sA[32][kLowK + 1], sB[32][kLowK + 1];
  int bi, bj;
  if (sym) {
    int t = blockIdx.x, len = tn;
    bi = 0;
    while (t >= len) {
      t -= len;
      ++bi;
      --len;
    }
    bj = bi + t;
  } else {
    bi = blockIdx.y;
    bj = blockIdx.x;
  }
  const int m0 = bi * 32, n0 = bj * 32;
  for (int idx = threadIdx.x; idx < 32 * K; idx += blockDim.x) {
    const int r = idx / K, k = idx - r * K;
    double va = 0.0, vb = 0.0;
    if (m0 + r < M) {
      va = A[(size_t)(m0 + r) * lda + k];
      if (s) va *= s[k];
    }
    if (n0 + r < N) vb = B[(size_t)(n0 + r) * ldb + k];
    sA[r][k] = va;
    sB[r][k] = vb;
  }
  __syncthreads();
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // column n0 + tx, rows m0 + ty + 8 q
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int k = 0; k < K; ++k) {
    const double vb = sB[tx][k];
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = fma(sA[ty + 8 * q][k], vb, acc[q]);
  }
  const int gn = n0 + tx;
  if (gn >= N) return;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int gm = m0 + ty + 8 * q;
    if (gm >= M || (sym && gn < gm)) continue;
    const double v = alpha * acc[q];
    double* cp = &C[(size_t)gm * ldc + gn];
    *cp = (beta == 0.0) ? v : v + beta * (*cp);
    if (sym && gn > gm) {
      double* cm = &C[(size_t)gn * ldc + gm];
      *cm = (beta == 0.0) ? v : v + beta * (*cm);
    }
  }
}

}  // namespace

void gemm_f64(cudaStream_t st, bool ta, bool tb, int M, int N, int K, double alpha,
              const double* A, int lda, const double* B, int ldb, const double* s, double beta,
              double* C, int ldc, int flags) {
  if (M <= 0 || N <= 0) return;
  if ((flags & G_SYM) && M != N) throw Error{KOT_ERR_INVALID, "gemm_f64: G_SYM needs M == N"};
  ProfScope ps(st, KC_GEMM_F64, 2.0 * gemm_macs(M, N, std::max(K, 0), flags),
               8.0 * ((double)M * K + (double)K * N + (double)M * N));
  if (K <= 0) {   // C = beta C
    if (beta == 0.0)
      for (int i = 0; i < M; ++i) KOT_CUDA(cudaMemsetAsync(C + (size_t)i * ldc, 0, N * sizeof(double), st));
    return;
  }
  if (K <= kLowK && !ta && tb && (flags & ~G_SYM) == 0) {
    const int tm = cdiv(M, 32), tn = cdiv(N, 32);
    const bool sym = (flags & G_SYM) != 0;
    const dim3 grid = sym ? dim3(tn * (tn + 1) / 2) : dim3(tn, tm);
    launch_pdl(k_gemm_f64_lowk, grid, dim3(256), 0, st, M, N, K, alpha, A, lda, B, ldb, s, beta, C, ldc,
               sym ? 1 : 0, tn);
    KOT_CHECK_LAUNCH();
    return;
  }
  int dev = 0, nsm = 0;
  KOT_CUDA(cudaGetDevice(&dev));
  KOT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  SkArgs a;
  a.M = M;
  a.N = N;
  a.K = K;
  a.flags = flags;
  a.alpha = alpha;
  a.beta = beta;
  a.A = A;
  a.B = B;
  a.s = s;
  a.C = C;
  a.lda = lda;
  a.ldb = ldb;
  a.ldc = ldc;
  const int tm = (M + SK_T - 1) / SK_T;
  a.tn = (N + SK_T - 1) / SK_T;
  a.ntiles = (flags & G_SYM) ? a.tn * (a.tn + 1) / 2 : tm * a.tn;
  long long T = 0;
  for (int t = 0; t < a.ntiles; ++t) {
    int m0, n0, kb, ke, len;
    sk_tile(flags, K, a.tn, t, m0, n0, kb, ke, len);
    T += len;
  }
  a.T = T;
  // two warps per SM sub-partition when each gets at least 32 k-steps, else one, else fewer
  // (W <= T keeps every share non-empty, which the arrival count relies on)
  if (T >= 32LL * SK_WARPS * nsm) a.W = SK_WARPS * nsm;
  else if (T >= 16LL * (SK_WARPS / 2) * nsm) a.W = (SK_WARPS / 2) * nsm;
  else a.W = (int)std::max<long long>(1, T / 16);
  {
    std::lock_guard<std::mutex> lk(g_sk_mu);
    SkWork& w = g_sk[{dev, st}];
    w.part.alloc((size_t)SK_WARPS * nsm * 2 * 256);
    if (w.cnt.n < (size_t)a.ntiles) {
      w.cnt.alloc((size_t)a.ntiles);
      KOT_CUDA(cudaMemsetAsync(w.cnt.p, 0, w.cnt.n * sizeof(unsigned), st));
    }
    a.part = w.part.p;
    a.cnt = w.cnt.p;
  }
  const int grid = std::min(nsm, a.W);   // warp w runs in CTA w mod grid
  if ((long long)grid * SK_WARPS < a.W) throw Error{KOT_ERR_INVALID, "gemm_f64: share count"};
  if (!ta && !tb) k_gemm_f64_sk<false, false><<<grid, 32 * SK_WARPS, 0, st>>>(a);
  else if (!ta && tb) k_gemm_f64_sk<false, true><<<grid, 32 * SK_WARPS, 0, st>>>(a);
  else if (ta && !tb) k_gemm_f64_sk<true, false><<<grid, 32 * SK_WARPS, 0, st>>>(a);
  else k_gemm_f64_sk<true, true><<<grid, 32 * SK_WARPS, 0, st>>>(a);
  KOT_CHECK_LAUNCH();
}

void coldot_upper(cudaStream_t st, int l, const double* R, const double* Y, double* out) {
  launch_pdl(k_coldot_upper, dim3(cdiv(l, 32)), dim3(32, 32), 0, st, l, R, Y, out);
  KOT_CHECK_LAUNCH();
}

void coldot_rows(cudaStream_t st, int rows, int n, const double* A, int lda, const double* Y, int ldy,
                 double scale, double* out) {
  if (n <= 0) return;
  launch_pdl(k_coldot_rows, dim3(cdiv(n, 32)), dim3(32, 32), 0, st, std::max(rows, 0), n, A, lda, Y, ldy,
             scale, out);
  KOT_CHECK_LAUNCH();
}

void gemv_f64(cudaStream_t st, int n, double alpha, const double* A, const double* x,
              double beta, double* y) {
  launch_pdl(k_gemv, dim3(cdiv((size_t)n * 32, 256)), dim3(256), 0, st, n, alpha, A, x, beta, y);
  KOT_CHECK_LAUNCH();
}

// Arrays up to kOneBlockN entries are reduced by one block in one launch.
constexpr size_t kOneBlockN = 1u << 14;

void dot_f64(cudaStream_t st, int n, const double* x, const double* y, double* out,
             double* partial) {
  if ((size_t)n <= kOneBlockN) {
    launch_pdl(k_dot_one, dim3(1), dim3(1024), 0, st, (size_t)n, x, y, out);
    KOT_CHECK_LAUNCH();
    return;
  }
  launch_pdl(k_dot_partial, dim3(kReduceBlocks), dim3(256), 0, st, (size_t)n, x, y, partial);
  launch_pdl(k_sum_partials, dim3(1), dim3(256), 0, st, kReduceBlocks, partial, out);
  KOT_LAUNCHED(2);
}

void sumsq_f64(cudaStream_t st, size_t n, const double* x, double* out, double* partial) {
  if (n <= kOneBlockN) {
    launch_pdl(k_dot_one, dim3(1), dim3(1024), 0, st, n, x, nullptr, out);
    KOT_CHECK_LAUNCH();
    return;
  }
  launch_pdl(k_dot_partial, dim3(kReduceBlocks), dim3(256), 0, st, n, x, nullptr, partial);
  launch_pdl(k_sum_partials, dim3(1), dim3(256), 0, st, kReduceBlocks, partial, out);
  KOT_LAUNCHED(2);
}

void cg_step(cudaStream_t st, int n, const double* Hp, double* p, double* x, double* e, double* sc, int cur,
             size_t nw, const double* Wp, double* W) {
  launch_pdl(k_cg_step, dim3(1), dim3(1024), 0, st, n, Hp, p, x, e, sc, cur, nw, Wp, W);
  KOT_CHECK_LAUNCH();
}

void two_norms(cudaStream_t st, size_t n1, const double* x, size_t n2, const double* a, const double* b,
               double* out2, double* partial) {
  const size_t n = std::max(n1, n2);
  if (n <= kOneBlockN / 4) {
    launch_pdl(k_two_norms, dim3(1), dim3(256), 0, st, n1, x, n2, a, b, out2);
    KOT_CHECK_LAUNCH();
    return;
  }
  const int nb = kReduceBlocks / 2;   // partial holds kReduceBlocks doubles: nb pairs
  launch_pdl(k_two_norms, dim3(nb), dim3(256), 0, st, n1, x, n2, a, b, partial);
  launch_pdl(k_sum_pairs, dim3(1), dim3(256), 0, st, nb, partial, out2);
  KOT_LAUNCHED(2);
}

void eig_norms(cudaStream_t st, size_t n1, const double* x, int rows, int cols, int ld, int nb,
               const double* A, const double* W, const double* base, double* out2, double* partial) {
  const size_t n = std::max(n1, (size_t)std::max(rows, 0) * std::max(cols, 0));
  if (rows <= 0 || cols <= 0) rows = cols = 0;
  if (n <= kOneBlockN / 4) {
    launch_pdl(k_eig_norms, dim3(1), dim3(256), 0, st, n1, x, rows, cols, ld, nb, A, W, base, out2);
    KOT_CHECK_LAUNCH();
    return;
  }
  const int nbk = kReduceBlocks / 2;   // partial holds kReduceBlocks doubles: nbk pairs
  launch_pdl(k_eig_norms, dim3(nbk), dim3(256), 0, st, n1, x, rows, cols, ld, nb, A, W, base, partial);
  launch_pdl(k_sum_pairs, dim3(1), dim3(256), 0, st, nbk, partial, out2);
  KOT_LAUNCHED(2);
}

void form_z(cudaStream_t st, int l, const double* X, const double* S, double a, double c, double* Z, double* FX) {
  launch_pdl(k_form_z, dim3(cdiv(l, 32), cdiv(l, 8)), dim3(32, 8), 0, st, l, X, S, a, c, Z, FX);
  KOT_CHECK_LAUNCH();
}

void grad_gamma_fused(cudaStream_t st, int n, double s, const double* Q, const double* gamma, const double* z,
                      const double* v, double* out) {
  launch_pdl(k_grad_gamma, dim3(cdiv((size_t)n * 32, 256)), dim3(256), 0, st, n, s, Q, gamma, z, v, out);
  KOT_CHECK_LAUNCH();
}

void sub_norms(cudaStream_t st, size_t n1, const double* x1, size_t n2, const double* X, const double* P,
               double* D, double* out2, double* partial) {
  const size_t n = std::max(n1, n2);
  if (n <= kOneBlockN / 4) {
    launch_pdl(k_sub_norms, dim3(1), dim3(256), 0, st, n1, x1, n2, X, P, D, out2);
    KOT_CHECK_LAUNCH();
    return;
  }
  const int nb = kReduceBlocks / 2;   // partial holds kReduceBlocks doubles: nb pairs
  launch_pdl(k_sub_norms, dim3(nb), dim3(256), 0, st, n1, x1, n2, X, P, D, partial);
  launch_pdl(k_sum_pairs, dim3(1), dim3(256), 0, st, nb, partial, out2);
  KOT_LAUNCHED(2);
}

void sum_pairs(cudaStream_t st, int nb, const double* partial, double* out2) {
  launch_pdl(k_sum_pairs, dim3(1), dim3(256), 0, st, nb, partial, out2);
  KOT_CHECK_LAUNCH();
}

void square_elems(cudaStream_t st, size_t n, const double* x, double* out) {
  launch_pdl(k_square, dim3(elementwise_grid(n)), dim3(256), 0, st, n, x, out);
  KOT_CHECK_LAUNCH();
}

void hmatvec(cudaStream_t st, int n, double alpha, const double* A, const double* x, double mu,
             const double* v, double* y) {
  launch_pdl(k_hmatvec, dim3(cdiv((size_t)n * 32, 256)), dim3(256), 0, st, n, alpha, A, x, mu, v, y);
  KOT_CHECK_LAUNCH();
}

void axpby(cudaStream_t st, size_t n, double a, const double* x, double b, const double* y,
           double* out) {
  launch_pdl(k_axpby, dim3(elementwise_grid(n)), dim3(256), 0, st, n, a, x, b, y, out);
  KOT_CHECK_LAUNCH();
}

void axpy_ratio(cudaStream_t st, size_t n, const double* num, const double* den, double sgn,
                const double* x, double* y, double* flag) {
  launch_pdl(k_axpy_ratio, dim3(elementwise_grid(n)), dim3(256), 0, st, n, num, den, sgn, x, y, flag);
  KOT_CHECK_LAUNCH();
}

void xpby_ratio(cudaStream_t st, size_t n, const double* x, const double* num, const double* den,
                double* y) {
  launch_pdl(k_xpby_ratio, dim3(elementwise_grid(n)), dim3(256), 0, st, n, x, num, den, y);
  KOT_CHECK_LAUNCH();
}

void fill(cudaStream_t st, size_t n, double v, double* out) {
  launch_pdl(k_fill, dim3(elementwise_grid(n)), dim3(256), 0, st, n, v, out);
  KOT_CHECK_LAUNCH();
}

void symmetrize(cudaStream_t st, int l, double* A) {
  launch_pdl(k_symmetrize, dim3(cdiv(l, 32), cdiv(l, 8)), dim3(32, 8), 0, st, l, A);
  KOT_CHECK_LAUNCH();
}

void add_diag(cudaStream_t st, int l, double v, double* A, int lda) {
  launch_pdl(k_add_diag, dim3(cdiv(l, 256)), dim3(256), 0, st, l, v, A, lda);
  KOT_CHECK_LAUNCH();
}

void copy_mat(cudaStream_t st, int rows, int cols, const double* A, int lda, double* B, int ldb) {
  if (rows <= 0 || cols <= 0) return;
  launch_pdl(k_copy_mat, dim3(cdiv(cols, 32), cdiv(rows, 8)), dim3(32, 8), 0, st, rows, cols, A, lda, B, ldb);
  KOT_CHECK_LAUNCH();
}

void sym_sum(cudaStream_t st, int l, const double* G, const double* S, double inv_mu,
             int complement, double* out) {
  launch_pdl(k_sym_sum, dim3(cdiv(l, 32), cdiv(l, 8)), dim3(32, 8), 0, st, l, G, S, inv_mu, complement, out);
  KOT_CHECK_LAUNCH();
}

}  // namespace kot
