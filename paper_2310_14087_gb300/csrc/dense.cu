// Dense FP64 building blocks: tiled GEMM with triangular k-range cuts, GEMV, deterministic
// reductions and elementwise helpers.
//
// FP64 on GB300 issues about two fused multiply-adds per clock per SM, so these kernels are
// bound by the FP64 pipe: the design goal is to keep all 152 SMs busy (small 32 x 32 tiles) and
// to skip work the triangular Cholesky factor makes zero, not to stage operands for tensor cores.
#include <algorithm>
#include <atomic>

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
  *a = get_event();
  KOT_CUDA(cudaEventRecord(*a, st));
}

void Profiler::end(cudaStream_t st, int cls, cudaEvent_t a, double fl, double by) {
  cudaEvent_t b = get_event();
  if (cudaEventRecord(b, st) != cudaSuccess) return;
  pending.push_back({cls, a, b, fl, by});
  if (pending.size() > 4096) collect();
}

void Profiler::collect() {
  for (auto& q : pending) {
    float t = 0.f;
    if (cudaEventSynchronize(q.b) == cudaSuccess && cudaEventElapsedTime(&t, q.a, q.b) == cudaSuccess) {
      launches[q.cls] += 1;
      ms[q.cls] += t;
      flops[q.cls] += q.flops;
      bytes[q.cls] += q.bytes;
    }
    pool.push_back(q.a);
    pool.push_back(q.b);
  }
  pending.clear();
}

void Profiler::reset() {
  collect();
  for (int i = 0; i < KC_COUNT; ++i) launches[i] = 0, ms[i] = flops[i] = bytes[i] = 0.0;
}

void Profiler::release() {
  collect();
  for (auto e : pool) cudaEventDestroy(e);
  pool.clear();
}

namespace {

constexpr int BK = 32, GT = 64;   // k-chunk and threads per CTA (8 x 8 thread grid)

// Tile BT x BT (32 or 16); each thread owns a (BT/8) x (BT/8) strided sub-block.  The 16 x 16
// variant is used when 32 x 32 tiles would leave most of the 152 SMs idle (l of a few hundred).
template <int BT, bool TA, bool TB>
__global__ void __launch_bounds__(GT) k_gemm_f64(int M, int N, int K, double alpha,
                                                 const double* __restrict__ A, int lda,
                                                 const double* __restrict__ B, int ldb,
                                                 const double* __restrict__ s, double beta,
                                                 double* __restrict__ C, int ldc, int flags) {
  constexpr int TT = BT / 8;
  const int m0 = blockIdx.y * BT, n0 = blockIdx.x * BT;
  if ((flags & G_SYM) && n0 < m0) return;
  __shared__ double As[BK][BT + 1];
  __shared__ double Bs[BK][BT + 1];
  int kbeg = 0, kend = K;
  if (flags & G_KLO_ROW) kbeg = max(kbeg, m0);
  if (flags & G_KLO_COL) kbeg = max(kbeg, n0);
  if (flags & G_KHI_COL) kend = min(kend, n0 + BT);
  if (flags & G_KHI_ROW) kend = min(kend, m0 + BT);
  const int t = threadIdx.x, tx = t & 7, ty = t >> 3;
  double acc[TT][TT];
#pragma unroll
  for (int i = 0; i < TT; ++i)
#pragma unroll
    for (int j = 0; j < TT; ++j) acc[i][j] = 0.0;

  for (int k0 = (kbeg / BK) * BK; k0 < kend; k0 += BK) {
#pragma unroll 4
    for (int r = 0; r < (BT * BK) / GT; ++r) {
      int idx = t + r * GT;
      int m, k;
      if (TA) { k = idx / BT; m = idx % BT; } else { m = idx / BK; k = idx % BK; }
      int gm = m0 + m, gk = k0 + k;
      double v = 0.0;
      if (gm < M && gk >= kbeg && gk < kend) {
        v = TA ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk];
        if (s) v *= s[gk];
      }
      As[k][m] = v;
    }
#pragma unroll 4
    for (int r = 0; r < (BT * BK) / GT; ++r) {
      int idx = t + r * GT;
      int n, k;
      if (TB) { n = idx / BK; k = idx % BK; } else { k = idx / BT; n = idx % BT; }
      int gn = n0 + n, gk = k0 + k;
      double v = 0.0;
      if (gn < N && gk >= kbeg && gk < kend)
        v = TB ? B[(size_t)gn * ldb + gk] : B[(size_t)gk * ldb + gn];
      Bs[k][n] = v;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < BK; ++k) {
      double a[TT], b[TT];
#pragma unroll
      for (int i = 0; i < TT; ++i) a[i] = As[k][ty + 8 * i];
#pragma unroll
      for (int j = 0; j < TT; ++j) b[j] = Bs[k][tx + 8 * j];
#pragma unroll
      for (int i = 0; i < TT; ++i)
#pragma unroll
        for (int j = 0; j < TT; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  const bool mirror = (flags & G_SYM) && n0 > m0;
#pragma unroll
  for (int i = 0; i < TT; ++i) {
    int gm = m0 + ty + 8 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < TT; ++j) {
      int gn = n0 + tx + 8 * j;
      if (gn >= N) continue;
      double v = alpha * acc[i][j];
      double* c = &C[(size_t)gm * ldc + gn];
      *c = (beta == 0.0) ? v : v + beta * (*c);
      if (mirror) {
        double* cm = &C[(size_t)gn * ldc + gm];
        *cm = (beta == 0.0) ? v : v + beta * (*cm);
      }
    }
  }
}

__global__ void k_coldot_upper(int l, const double* __restrict__ R, const double* __restrict__ Y,
                               double* __restrict__ out) {
  __shared__ double part[8][33];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i = blockIdx.x * 32 + tx;
  double acc = 0.0;
  if (i < l)
    for (int a = ty; a <= i; a += 8) acc = fma(R[(size_t)a * l + i], Y[(size_t)a * l + i], acc);
  part[ty][tx] = acc;
  __syncthreads();
  if (ty == 0 && i < l) {
    double s = 0.0;
#pragma unroll
    for (int r = 0; r < 8; ++r) s += part[r][tx];
    out[i] = s;
  }
}

__global__ void k_gemv(int n, double alpha, const double* __restrict__ A,
                       const double* __restrict__ x, double beta, double* __restrict__ y) {
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
  __shared__ double sh[256];
  double acc = 0.0;
  for (size_t i = blockIdx.x * 256 + threadIdx.x; i < n; i += (size_t)gridDim.x * 256)
    acc = fma(x[i], y ? y[i] : x[i], acc);
  double s = block_sum<256>(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void k_sum_partials(int nb, const double* __restrict__ partial, double* __restrict__ out) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nb; i += 256) acc += partial[i];
  double s = block_sum<256>(acc, sh);
  if (threadIdx.x == 0) *out = s;
}

__global__ void k_axpby(size_t n, double a, const double* __restrict__ x, double b,
                        const double* __restrict__ y, double* __restrict__ out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    double v = a * x[i];
    if (y) v = fma(b, y[i], v);
    out[i] = v;
  }
}

__global__ void k_fill(size_t n, double v, double* __restrict__ out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    out[i] = v;
}

__global__ void k_symmetrize(int l, double* A) {
  const int j = blockIdx.x * 32 + threadIdx.x, i = blockIdx.y * 8 + threadIdx.y;
  if (i < l && j < l && i < j) {
    double v = 0.5 * (A[(size_t)i * l + j] + A[(size_t)j * l + i]);
    A[(size_t)i * l + j] = v;
    A[(size_t)j * l + i] = v;
  }
}

__global__ void k_add_diag(int l, double v, double* A, int lda) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < l) A[(size_t)i * lda + i] += v;
}

__global__ void k_copy_mat(int rows, int cols, const double* __restrict__ A, int lda,
                           double* __restrict__ B, int ldb) {
  const int j = blockIdx.x * 32 + threadIdx.x, i = blockIdx.y * 8 + threadIdx.y;
  if (i < rows && j < cols) B[(size_t)i * ldb + j] = A[(size_t)i * lda + j];
}

__global__ void k_sym_sum(int l, const double* __restrict__ G, const double* __restrict__ S,
                          double inv_mu, int complement, double* __restrict__ out) {
  const int j = blockIdx.x * 32 + threadIdx.x, i = blockIdx.y * 8 + threadIdx.y;
  if (i >= l || j >= l) return;
  double g = G[(size_t)i * l + j] + G[(size_t)j * l + i];
  out[(size_t)i * l + j] = complement ? fma(inv_mu, S[(size_t)i * l + j], -g) : g;
}

inline int cdiv(size_t a, int b) { return (int)((a + b - 1) / b); }

}  // namespace

void gemm_f64(cudaStream_t st, bool ta, bool tb, int M, int N, int K, double alpha,
              const double* A, int lda, const double* B, int ldb, const double* s, double beta,
              double* C, int ldc, int flags) {
  if (M <= 0 || N <= 0) return;
  // 32 x 32 tiles unless that gives fewer CTAs than about two per SM
  const bool small = (size_t)cdiv(N, 32) * cdiv(M, 32) < 2 * 152;
  const int BT = small ? 16 : 32;
  dim3 grid(cdiv(N, BT), cdiv(M, BT));
  ProfScope ps(st, KC_GEMM_F64, 2.0 * M * N * (double)K, 8.0 * ((double)M * K + (double)K * N + (double)M * N));
  if (K <= 0) {   // C = beta C
    if (beta == 0.0)
      for (int i = 0; i < M; ++i) KOT_CUDA(cudaMemsetAsync(C + (size_t)i * ldc, 0, N * sizeof(double), st));
    return;
  }
#define KOT_GEMM_LAUNCH(BTV)                                                                      \
  if (!ta && !tb) k_gemm_f64<BTV, false, false><<<grid, GT, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, s, beta, C, ldc, flags); \
  else if (!ta && tb) k_gemm_f64<BTV, false, true><<<grid, GT, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, s, beta, C, ldc, flags); \
  else if (ta && !tb) k_gemm_f64<BTV, true, false><<<grid, GT, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, s, beta, C, ldc, flags); \
  else k_gemm_f64<BTV, true, true><<<grid, GT, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, s, beta, C, ldc, flags);
  if (small) {
    KOT_GEMM_LAUNCH(16)
  } else {
    KOT_GEMM_LAUNCH(32)
  }
#undef KOT_GEMM_LAUNCH
  KOT_CHECK_LAUNCH();
}

void coldot_upper(cudaStream_t st, int l, const double* R, const double* Y, double* out) {
  k_coldot_upper<<<cdiv(l, 32), dim3(32, 8), 0, st>>>(l, R, Y, out);
  KOT_CHECK_LAUNCH();
}

void gemv_f64(cudaStream_t st, int n, double alpha, const double* A, const double* x,
              double beta, double* y) {
  k_gemv<<<cdiv((size_t)n * 32, 256), 256, 0, st>>>(n, alpha, A, x, beta, y);
  KOT_CHECK_LAUNCH();
}

void dot_f64(cudaStream_t st, int n, const double* x, const double* y, double* out,
             double* partial) {
  k_dot_partial<<<kReduceBlocks, 256, 0, st>>>((size_t)n, x, y, partial);
  k_sum_partials<<<1, 256, 0, st>>>(kReduceBlocks, partial, out);
  KOT_LAUNCHED(2);
}

void sumsq_f64(cudaStream_t st, size_t n, const double* x, double* out, double* partial) {
  k_dot_partial<<<kReduceBlocks, 256, 0, st>>>(n, x, nullptr, partial);
  k_sum_partials<<<1, 256, 0, st>>>(kReduceBlocks, partial, out);
  KOT_LAUNCHED(2);
}

void axpby(cudaStream_t st, size_t n, double a, const double* x, double b, const double* y,
           double* out) {
  k_axpby<<<std::min(cdiv(n, 256), 1216), 256, 0, st>>>(n, a, x, b, y, out);
  KOT_CHECK_LAUNCH();
}

void fill(cudaStream_t st, size_t n, double v, double* out) {
  k_fill<<<std::min(cdiv(n, 256), 1216), 256, 0, st>>>(n, v, out);
  KOT_CHECK_LAUNCH();
}

void symmetrize(cudaStream_t st, int l, double* A) {
  k_symmetrize<<<dim3(cdiv(l, 32), cdiv(l, 8)), dim3(32, 8), 0, st>>>(l, A);
  KOT_CHECK_LAUNCH();
}

void add_diag(cudaStream_t st, int l, double v, double* A, int lda) {
  k_add_diag<<<cdiv(l, 256), 256, 0, st>>>(l, v, A, lda);
  KOT_CHECK_LAUNCH();
}

void copy_mat(cudaStream_t st, int rows, int cols, const double* A, int lda, double* B, int ldb) {
  if (rows <= 0 || cols <= 0) return;
  k_copy_mat<<<dim3(cdiv(cols, 32), cdiv(rows, 8)), dim3(32, 8), 0, st>>>(rows, cols, A, lda, B, ldb);
  KOT_CHECK_LAUNCH();
}

void sym_sum(cudaStream_t st, int l, const double* G, const double* S, double inv_mu,
             int complement, double* out) {
  k_sym_sum<<<dim3(cdiv(l, 32), cdiv(l, 8)), dim3(32, 8), 0, st>>>(l, G, S, inv_mu, complement, out);
  KOT_CHECK_LAUNCH();
}

}  // namespace kot
