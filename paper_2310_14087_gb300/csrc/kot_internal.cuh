// Internal declarations shared by the CUDA translation units of libkot.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "../../include/kot.h"

namespace kot {

// ------------------------------------------------------------------ error plumbing
struct Error {
  kot_status status;
  std::string what;
};

#define KOT_CUDA(call)                                                                    \
  do {                                                                                    \
    cudaError_t e__ = (call);                                                             \
    if (e__ != cudaSuccess)                                                               \
      throw ::kot::Error{e__ == cudaErrorMemoryAllocation ? KOT_ERR_OOM : KOT_ERR_CUDA,    \
                         std::string(#call) + ": " + cudaGetErrorString(e__)};            \
  } while (0)

// Every kernel launch site is followed by KOT_LAUNCHED(k) with the number of kernels it just
// launched; the running total is readable through kot_launch_count().
void note_launches(long long k);
long long launch_total();
#define KOT_LAUNCHED(k)                   \
  do {                                    \
    ::kot::note_launches(k);              \
    KOT_CUDA(cudaPeekAtLastError());      \
  } while (0)
#define KOT_CHECK_LAUNCH() KOT_LAUNCHED(1)

// ------------------------------------------------------------------ programmatic dependent launch
// A kernel launched by launch_pdl may be scheduled while its predecessor in the stream is still
// running (programmatic stream serialisation, sm_90 and later).  Such a kernel calls pdl_wait()
// before its first global-memory access and before any early exit: the wait returns once every
// prerequisite grid has completed with its writes visible, and a grid that cannot complete
// before its own wait returned keeps completion ordered along the stream.  pdl_trigger() after
// the wait lets the successor's CTAs be scheduled onto free SMs while this grid runs.  Both
// instructions are no-ops in a kernel launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Programmatic launches are on unless the environment sets KOT_PDL=0 (read once per process),
// e.g. for a profiler run that should see the plain stream-ordered launches.
bool pdl_enabled();

template <typename... KArgs, typename... Args>
void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  KOT_CUDA(cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...));
}

// ------------------------------------------------------------------ launch profiler
// Kernel classes the profiler can time (kot_kernel_class in kot.h uses the same numbering).
enum KClass : int {
  KC_GEMM_F64 = 0,      // k_gemm_f64
  KC_JACOBI = 1,        // k_jacobi_coop (all sweeps of one decomposition, FP64)
  KC_RESERVED_2 = 2,    // unused (kept so that the class numbers of kot.h stay stable)
  KC_EMBED = 3,         // k_embed, k_potential (kernel sums over samples)
  KC_PAIRS = 4,         // k_pair_tiles
  KC_GRAM = 5,          // k_gram
  KC_CHOL = 6,          // Cholesky diagonal / panel kernels
  KC_GEMM_TC = 7,       // k_tc_gemm_bf16 (tcgen05 tensor-core GEMM)
  KC_REFINE = 8,        // k_refine_correction (eigenbasis refinement step; its products are
                        // counted as gemm_f64 or gemm_oz)
  KC_GEMM_OZ = 9,       // k_oz_gemm (FP64-accurate products emulated on the tensor cores)
  KC_OZ_AUX = 10,       // slicing (k_oz_split_cluster, or k_oz_rowexp + k_oz_split) and k_oz_finalize
  KC_MATVEC = 11,       // one Schur-operator application of CG (all its launches, Algorithm 1)
  KC_COUNT = 12
};

// When a profiler is installed for the calling thread, instrumented launch sites record a CUDA
// event pair around each launch of an enabled class together with the launch's algorithmic
// flop and byte counts and the flops it executes (e.g. an FP64-accurate product of 2MNK flops
// executes 2MNK per BF16 slice pair); collect() waits for the events and accumulates per class.
struct Profiler {
  int mask = 0;
  int every = 1;                       // time one launch in `every` of each enabled class
  long long seen[KC_COUNT] = {};       // launches of each enabled class since the last reset
  struct Pending { int cls; cudaEvent_t a, b; double flops, bytes, exec; };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  long launches[KC_COUNT] = {};
  double ms[KC_COUNT] = {}, flops[KC_COUNT] = {}, bytes[KC_COUNT] = {}, exec[KC_COUNT] = {};
  std::mutex mu;                       // the solver's two host threads share one profiler
  bool on(int cls) const { return (mask >> cls) & 1; }
  // enabled, and this launch is one of the sampled ones
  bool take(int cls) {
    std::lock_guard<std::mutex> lk(mu);
    return on(cls) && (seen[cls]++ % every) == 0;
  }
  cudaEvent_t get_event();
  void begin(cudaStream_t st, int cls, cudaEvent_t* a);
  void end(cudaStream_t st, int cls, cudaEvent_t a, double fl, double by, double ex);
  void collect();
  void reset();
  void release();
 private:
  void collect_locked();
};
Profiler* current_profiler();
void set_current_profiler(Profiler* p);

// RAII helper around one launch: `ProfScope ps(st, KC_x, flops, bytes[, executed flops]); launch...;`
struct ProfScope {
  Profiler* p;
  cudaStream_t st;
  int cls;
  double fl, by, ex;
  cudaEvent_t a = nullptr;
  ProfScope(cudaStream_t s, int c, double f, double b, double e = -1.0)
      : p(current_profiler()), st(s), cls(c), fl(f), by(b), ex(e < 0.0 ? f : e) {
    if (p && p->take(cls)) p->begin(st, cls, &a);
    else p = nullptr;
  }
  ~ProfScope() {
    if (p) p->end(st, cls, a, fl, by, ex);
  }
};

// ------------------------------------------------------------------ device buffers
template <typename T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  void alloc(size_t count) {
    if (count <= n) return;
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
    KOT_CUDA(cudaMalloc(&p, count * sizeof(T)));
    n = count;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
};

// ------------------------------------------------------------------ dense kernels (dense.cu)
// GEMM flags: which operand is triangular, so the k-range of a tile can be cut.
enum GemmFlags : int {
  G_KLO_ROW = 1,   // opA(A)[m,k] == 0 for k < m   (opA(A) upper triangular)
  G_KLO_COL = 2,   // opB(B)[k,n] == 0 for k < n   (opB(B) lower triangular)
  G_KHI_COL = 4,   // opB(B)[k,n] == 0 for k > n   (opB(B) upper triangular)
  G_KHI_ROW = 8,   // opA(A)[m,k] == 0 for k > m   (opA(A) lower triangular)
  G_SYM = 16       // result is symmetric: compute tiles with n0 >= m0, mirror the rest
};

// C[M,N] = alpha * sum_k opA(A)[m,k] * s[k] * opB(B)[k,n] + beta * C
//   opA(A) = A (M x K, lda) or A^T (A stored K x M, lda) ; same for B (K x N or N x K).
void gemm_f64(cudaStream_t st, bool ta, bool tb, int M, int N, int K, double alpha,
              const double* A, int lda, const double* B, int ldb, const double* s, double beta,
              double* C, int ldc, int flags);

// out[i] = sum_a R[a,i] * Y[a,i] for a <= i  (Phi(X) = diag(R^T X R) with Y = X R)
void coldot_upper(cudaStream_t st, int l, const double* R, const double* Y, double* out);

// out[i] = scale * sum_{a < rows} A[a,i] * Y[a,i], i < n (row-major, leading dimensions lda, ldy)
void coldot_rows(cudaStream_t st, int rows, int n, const double* A, int lda, const double* Y, int ldy,
                 double scale, double* out);

// y = alpha * A x + beta * y (A: n x n row-major)
void gemv_f64(cudaStream_t st, int n, double alpha, const double* A, const double* x,
              double beta, double* y);

// Deterministic reductions.  Results land in device memory (one double).
void dot_f64(cudaStream_t st, int n, const double* x, const double* y, double* out,
             double* partial);
// out = sum x^2 over a n-element array
void sumsq_f64(cudaStream_t st, size_t n, const double* x, double* out, double* partial);
constexpr int kReduceBlocks = 128;   // size of the partial buffer the reductions need
// One CG step with device-resident scalars (see k_cg_step in dense.cu): sc[5 + cur] = |e|^2 in,
// sc[3] = p.Hp, sc[5 + (cur ^ 1)] = new |e|^2, sc[7] = 1 on non-positive curvature; W (nw
// entries, may be null) += (step length) Wp alongside x.
void cg_step(cudaStream_t st, int n, const double* Hp, double* p, double* x, double* e, double* sc, int cur,
             size_t nw = 0, const double* Wp = nullptr, double* W = nullptr);
// out2[0] = |x|^2 (n1 entries), out2[1] = |a - b|^2 (n2 entries); partial: kReduceBlocks doubles
void two_norms(cudaStream_t st, size_t n1, const double* x, size_t n2, const double* a, const double* b,
               double* out2, double* partial);
// Norms of the CG stopping test in the eigenbasis: out2[0] = |x|^2 (n1 entries) and
// out2[1] = (base ? *base : 0) + sum_{r < rows, j < cols} w_j (A[r,j] - c_j W[r,j])^2 with
// (w_j, c_j) = (2, 1) for j < nb and (1, 2) for j >= nb; W may be null (zero).  partial:
// kReduceBlocks doubles.
void eig_norms(cudaStream_t st, size_t n1, const double* x, int rows, int cols, int ld, int nb,
               const double* A, const double* W, const double* base, double* out2, double* partial);
// Complement form of the same test (Sec. 4.3, last paragraph): out2[0] = |x|^2 (l entries),
// out2[1] = ||A2 - Psi o Vx||_F^2 from the alpha-bar rows U of Vx = Cb diag(x) Cb^T (nb x l, ld l),
// A2 (l x l), KK = Kt o Kt, phi_at2 = Phi(at2) and *base = ||A2||_F^2 (see k_eig_norms_comp).
void eig_norms_comp(cudaStream_t st, int l, const double* x, int nb, const double* sig, double mu,
                    const double* A2, const double* U, const double* KK, const double* phi_at2,
                    const double* base, double* out2, double* partial);
// Z = sym(X - a S) - c I (S null: zero); FX (may be null) = S + c I.  l x l, row-major.
void form_z(cudaStream_t st, int l, const double* X, const double* S, double a, double c, double* Z, double* FX);
// out = s Q gamma - s z - v (Q: n x n)
void grad_gamma_fused(cudaStream_t st, int n, double s, const double* Q, const double* gamma, const double* z,
                      const double* v, double* out);
// D = X - P over n2 entries; out2[0] = |x1|^2 (n1 entries), out2[1] = |D|^2; partial: kReduceBlocks doubles
void sub_norms(cudaStream_t st, size_t n1, const double* x1, size_t n2, const double* X, const double* P,
               double* D, double* out2, double* partial);
// out2 = the column sums of nb (s1, s2) pairs in partial
void sum_pairs(cudaStream_t st, int nb, const double* partial, double* out2);
// out[i] = x[i]^2 (out may alias x)
void square_elems(cudaStream_t st, size_t n, const double* x, double* out);
// y = alpha A x + mu x + v (v may be null)
void hmatvec(cudaStream_t st, int n, double alpha, const double* A, const double* x, double mu,
             const double* v, double* y);

// Elementwise helpers.
void axpby(cudaStream_t st, size_t n, double a, const double* x, double b, const double* y,
           double* out);                                           // out = a x + b y
void fill(cudaStream_t st, size_t n, double v, double* out);
// Step-length updates with device-resident scalars (no host round trip inside CG):
// y += sgn (num/den) x, or -- if den <= 0 -- nothing and *flag = 1;  y = x + (num/den) y.
void axpy_ratio(cudaStream_t st, size_t n, const double* num, const double* den, double sgn,
                const double* x, double* y, double* flag);
void xpby_ratio(cudaStream_t st, size_t n, const double* x, const double* num, const double* den,
                double* y);
void symmetrize(cudaStream_t st, int l, double* A);                // A = (A + A^T)/2
void add_diag(cudaStream_t st, int l, double v, double* A, int lda);
void copy_mat(cudaStream_t st, int rows, int cols, const double* A, int lda, double* B, int ldb);
// out = G + G^T (sign = +1) or S/mu - (G + G^T) (sign = -1, S given)
void sym_sum(cudaStream_t st, int l, const double* G, const double* S, double inv_mu,
             int complement, double* out);

// ------------------------------------------------------------------ features (features.cu)
void embed_f64(cudaStream_t st, int n, int d, int l, const double* S, const double* P,
               double inv2s2, double* w);                          // w_i = mean_j k(s_j, p_i)
// sum_ij k(s_i, s_j) / n^2 into *out (partial: kPairBlocks doubles)
void pair_mean_f64(cudaStream_t st, int n, int d, const double* S, double inv2s2, double* out,
                   double* partial, int partial_cap);
int pair_blocks(int n);                                            // partials the above needs
// u(x_q), grad u(x_q), T(x_q) = x_q - grad u(x_q) at m query points Pq (m x d) from samples S
// (n x d), filling points Sf (l x d) and dual weights gamma (any output may be null)
void potential_f64(cudaStream_t st, int m, int d, int n, const double* S, int l, const double* Sf,
                   const double* gamma, const double* Pq, double sigma, double lambda2, double* u,
                   double* grad, double* tmap);
// fp32: the distances and exponentials of Q and K in FP32 (k_gram_f32), else FP64
void gram_f64(cudaStream_t st, int l, int d, const double* Xf, const double* Yf, double inv2s2,
              double lambda2, const double* w_mu, const double* w_nu, double* Q, double* K,
              double* c, double* z, bool fp32 = false);
// c_i = ||xf_i - yf_i||^2, z_i = w_mu_i + w_nu_i - lambda2 c_i (the cost and dual vector of Sec. 3)
void cost_z_f64(cudaStream_t st, int l, int d, const double* Xf, const double* Yf, double lambda2,
                const double* w_mu, const double* w_nu, double* c, double* z);
// Upper Cholesky of A + eps I in place (A: l x l, only the upper triangle is read).  The lower
// triangle is zeroed.  *info (device int) = 0 on success, j+1 if pivot j was not positive.
void zero_lower(cudaStream_t st, int l, double* A);        // A[i][j] = 0 for j < i
void cholesky_upper_f64(cudaStream_t st, int l, double* A, double eps, int* info);
// bound for the EG step (see kot_options.eg_step): out[0] = max rowsum |Q|, out[1] = max rowsum
// of (R^T R)_ij^2 given Kt = R^T R.
void rowsum_bounds(cudaStream_t st, int l, const double* Q, const double* Kt, double* out2);

// ------------------------------------------------------------------ eigen (eig.cu)
struct OzWork;
struct JacobiWork {
  OzWork* oz = nullptr;     // non-null: the eigensolver's products are emulated FP64 (tensor cores)
  // a refinement step whose correction is at most this is the last one (the basis it leaves is
  // accurate to about refine_done^2); 1e-8 leaves FP64 rounding
  double refine_done = 1e-8;
  DevBuf<double> A, V;      // A: two lp x lp buffers; V: lp x lp
  DevBuf<double> rot;       // two rounds x lp/2 pairs x (c, s)
  DevBuf<int> pairs;        // lp
  DevBuf<int> rank;         // l
  DevBuf<double> eye;       // l x l identity: G of the first step of a refinement without a warm basis
  DevBuf<double> X0;        // I + E after that step, the start of the rest
  DevBuf<double> B32;       // l x l basis from the shared-memory FP32 Jacobi (l <= 160)
  int eye_l = 0;
  DevBuf<double> partial, scal;
  DevBuf<unsigned> bar;     // grid barrier [arrivals, generation]
  DevBuf<int> flags;        // [error, 2 * sweeps + final buffer]
  // refinement of a warm basis (l x l each, ld l): ping-pong bases, Z X, X^T Z X, X^T X, I + E
  DevBuf<double> Xa, Xb, Y, S, G, F, lam;
  DevBuf<unsigned long long> mx;   // [max |E_ij| (i != j), max |I - X^T X|] as ordered bits, count of lambda <= 0
  int threads_override = 0;        // > 0: threads per CTA of the Jacobi kernel (the autotuner's probes)
  int last_sweeps = 0;             // Jacobi sweeps of the last call
  int last_refine = 0;             // refinement steps of the last call (0: Jacobi was used)
  bool last_trivial = false;       // no start basis, and Z was diagonal to the tolerance
  int last_nb = -1;                // eigenvalues <= 0 of a refined decomposition (-1: not counted)
  void release() {
    for (DevBuf<double>* b : {&A, &V, &rot, &partial, &scal, &Xa, &Xb, &Y, &S, &G, &F, &lam, &eye, &X0, &B32}) b->release();
    eye_l = 0;
    pairs.release();
    rank.release();
    bar.release();
    flags.release();
    mx.release();
  }
};

// Symmetric eigen-decomposition Z = P diag(sig) P^T, sig ascending.  Z: l x l (full
// symmetric, read only).  If warm != nullptr its columns (an orthogonal l x l basis, row-major)
// are used as the starting basis.  P: l x l output (row-major, column j = eigenvector j).
// With a warm basis the decomposition is first refined from it (at most max_refine steps of
// the Ogita-Aishima iteration, GEMMs only); if that does not converge quickly, from warm2 (an
// alternative basis, may alias P) when given, and failing both it is rebuilt by Jacobi sweeps
// from warm.  w.last_sweeps / w.last_refine report which ran.
// Returns the number of sweeps taken; throws on non-convergence within max_sweeps.
// ctas: CTAs of the cooperative launch (0 = one per SM).
int eig_sym_f64(cudaStream_t st, int l, const double* Z, const double* warm, double* P,
                double* sig, JacobiWork& w, int max_sweeps, double* host_scal, int ctas,
                int max_refine, const double* warm2 = nullptr);

// ------------------------------------------------------------------ tensor cores (tc_gemm.cu)
// Logical operand of C = alpha op(A) op(B)^T + beta C: element (r, k) is
// (trans ? src[k * ld + r] : src[r * ld + k]) * (scale ? scale[k] : 1).
struct TcOperand {
  const double* src;
  int ld;
  bool trans;
  const double* scale;
};
struct TcWork {
  DevBuf<unsigned short> a, b;   // BF16 split operands
  DevBuf<int> err;               // set by a CTA whose bounded wait gave up
};
// C (M x N, FP64, ldc) = alpha * sum_k opA(r=m, k) opB(r=n, k) + beta * C with K-length rows,
// on tcgen05 tensor cores with each operand split into `pieces` BF16 terms (1..3).
void gemm_tc(cudaStream_t st, TcWork& w, int M, int N, int K, const TcOperand& A,
             const TcOperand& B, int pieces, double alpha, double beta, double* C, int ldc);
// Nonzero if a tensor-core GEMM CTA timed out since the last call (clears the flag).
int gemm_tc_error(cudaStream_t st, TcWork& w);
// Launch a kernel whose bounded mbarrier wait nothing completes (polls >= 1); returns the
// error flag it leaves (1: the wait gave up, as it must).
int starved_wait_probe(cudaStream_t st, TcWork& w, long long polls);

// ------------------------------------------------------------------ FP64 emulation (oz_gemm.cu)
// FP64-accurate C (M x N, ldc) = alpha * sum_k opA(r=m, k) opB(r=n, k) + beta * C on the tensor
// cores: every operand row is cut into `slices` (3..8) fixed-point BF16 slices whose products
// are summed exactly in FP32 and combined in float-float (error about 2^-(8 slices - 1) relative to
// max|A row| max|B row| K).  sym: the result is symmetric (M == N); it is made exactly so.
struct OzWork {
  DevBuf<unsigned short> a, b;   // sliced operands
  DevBuf<int> part;              // per-row exponent partials
  DevBuf<double> fac;            // per-row scale factors
  DevBuf<float2> w;              // per-split partial sums
  DevBuf<int> err;               // set by a CTA whose bounded wait gave up
  int slices = 6;
  int splits_override = 0;       // > 0: use this split count (the autotuner's probes)
  int bn_override = 0;           // 64 or 128: use this output-tile width (the autotuner's probes)
  // gemm_acc sends products of fewer multiply-add flops (2 M N K, halved for a symmetric result)
  // to the FP64 GEMM: below about this size the three launches of the emulated product cost
  // more than the FP64 pipes need for the whole product (kot_options.tc_min_flops)
  double f64_below = 8e6;
  // last TMA descriptors (CUtensorMap, 128 bytes) and the (buffer, rows, cols) they describe
  alignas(64) unsigned char map_a[128], map_b[128];
  const void* key_a = nullptr;
  const void* key_b = nullptr;
  int rows_a = 0, cols_a = 0, rows_b = 0, cols_b = 0, box_b = 0;
  void release() {
    a.release();
    b.release();
    part.release();
    fac.release();
    w.release();
    err.release();
  }
};
void gemm_oz(cudaStream_t st, OzWork& w, int M, int N, int K, const TcOperand& A, const TcOperand& B,
             int slices, double alpha, double beta, double* C, int ldc, bool sym);
int gemm_oz_error(cudaStream_t st, OzWork& w);
// Autotuner table: split count of the emulated product per device, size bucket of max(M, N)
// (ceil log2) and slice count (0 = not tuned, use the occupancy rule).
int tuned_splits(int dev, int mn, int slices);
void set_tuned_splits(int dev, int mn, int slices, int splits);
int tuned_tile_width(int dev, int mn, int slices);   // 64, 128 or 0 (not tuned)
void set_tuned_tile_width(int dev, int mn, int slices, int bn);
// Autotuner table for the cooperative Jacobi eigensolver: CTAs per size bucket (0 = one per SM).
int tuned_jacobi_ctas(int dev, int l);
void set_tuned_jacobi_ctas(int dev, int l, int ctas);
// ... and its threads per CTA (256, 512 or 1024; 0 = not tuned, 512)
int tuned_jacobi_threads(int dev, int l);
void set_tuned_jacobi_threads(int dev, int l, int threads);
// gemm_f64's interface (C = alpha opA(A) diag(s) opB(B) + beta C, triangular/symmetric flags):
// on the FP64 pipes when oz is null, else emulated on the tensor cores with oz->slices slices
// (the triangular flags only cut work on the FP64 pipes; G_SYM is honoured by both).
void gemm_acc(cudaStream_t st, OzWork* oz, bool ta, bool tb, int M, int N, int K, double alpha,
              const double* A, int lda, const double* B, int ldb, const double* s, double beta,
              double* C, int ldc, int flags);

// ------------------------------------------------------------------ Newton pieces (newton.cu)
// V = weights o U for the rows of the G + G^T form of T (|alpha| rows: columns in alpha by 1/(2 mu),
// columns in alpha-bar by xi) or of the complement form (|alpha-bar| rows: 1/(2 mu) on alpha-bar,
// 1/mu - xi on alpha).  U null: in place on V.  See t_apply and schur_eig in kot_api.cu.
void t_weights(cudaStream_t st, int l, int nb, const double* sig, double mu, int complement,
               double* V, const double* U = nullptr);
// The Schur operator's rows and columns for few carried rows (crow <= 32; see newton.cu):
// carry/W (crow x l) from rows r0.. of Cb and p; Hp = alpha H p + mu p + c diag(Cb_rows^T W Cb).
constexpr int kSkinnyRows = 32;
void schur_rows(cudaStream_t st, int l, int crow, int r0, const double* Cb, const double* p, const double* sig,
                double mu, int nb, int complement, double* carry, double* W);
void schur_cols(cudaStream_t st, int l, int crow, int r0, const double* CbT, const double* W, double c,
                const double* H, double alpha, const double* p, double mu, double* Hp);
void transpose(cudaStream_t st, int l, const double* A, double* B);   // B = A^T (l x l)
// D = A2 - Psi o Vx (l x l): the eigenbasis form of dX = at2 - T[Phi*(x)] from the full Vx.
void assemble_psi(cudaStream_t st, int l, int nb, const double* sig, double mu, const double* A2,
                  const double* Vx, double* D);
// Right-hand side of Algorithm 1 in the eigenbasis: A2 = -(1 + Psi) o B/(mu + 1) for B = P^T r2 P
// (l x l), i.e. A2 = P^T at2 P.
void rhs_weights(cudaStream_t st, int l, int nb, const double* sig, double mu, const double* B, double* A2);
// D = A2 - P^T T[Phi*(x)] P with T[Phi*(x)] given by its alpha rows Wx (alpha x alpha halved).
void assemble_dir(cudaStream_t st, int l, int nb, const double* A2, const double* Wx, double* D);
// Count of eigenvalues <= 0 in sorted sig (device) -> *nb (device int)
void count_nonpos(cudaStream_t st, int l, const double* sig, int* nb);

}  // namespace kot
