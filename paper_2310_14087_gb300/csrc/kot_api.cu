// C ABI of libkot and the host-side driver of Algorithm 2.  Every arithmetic step runs in the
// kernels of dense.cu, features.cu, eig.cu and newton.cu; the host only sequences launches,
// reads back the scalars that steer the iteration (norms, CG step lengths, the alpha split) and
// applies the scalar rules of Algorithm 2 (theta update, acceptance, stopping).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>
#include <atomic>
#include <condition_variable>
#include <exception>
#include <mutex>
#include <numeric>
#include <thread>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "kot_internal.cuh"

using namespace kot;

namespace {
// NVTX range for the phases of a solve (visible to Nsight tools, free otherwise)
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};
}  // namespace

// layouts the ctypes binding mirrors (LP64, natural alignment)
static_assert(sizeof(kot_options) == 184, "kot_options layout");
static_assert(sizeof(kot_result) == 96, "kot_result layout");

namespace {

struct EigSlot {
  DevBuf<double> P, sig;
  int nb = 0;          // number of eigenvalues <= 0 (alpha-bar); alpha = the last l - nb
  bool valid = false;
  bool trivial = false;   // came from an exactly diagonal matrix (identity basis): no use as a warm start
};

struct ResState {
  DevBuf<double> r1, r2;
  double n1 = 0, n2 = 0, norm = 0;
};

__global__ void k_maxdiag(int l, const double* __restrict__ K, double* __restrict__ out) {
  __shared__ double sh[256];
  double m = -INFINITY;
  for (int i = threadIdx.x; i < l; i += 256) m = fmax(m, K[(size_t)i * l + i]);
  sh[threadIdx.x] = m;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

}  // namespace

struct kot_ctx {
  kot_options opt{};
  cudaStream_t st = nullptr;
  bool own_stream = false;
  std::string err = "no error";
  int l = 0;
  bool have = false;
  double lambda1 = 0, lambda2 = 0, q2 = 0, eps = 0, eg_L = 0;
  DevBuf<double> Q, K, R, z, w_mu, w_nu, c;
  // samples and filling points of the last kot_build_features (for kot_potentials)
  DevBuf<double> sX, sY, sXf, sYf;
  int d = 0, n = 0;
  double sigma = 0;
  bool have_samples = false;
  DevBuf<double> stage[8];                     // host-pointer mode staging
  DevBuf<double> g, X, vg, vX, tg, tX, dg, dX;
  ResState rw, rv, rt;
  EigSlot ew, ev, et, e1, e2;
  DevBuf<double> M1, M2, M3, M4, M5, M6, TU, TV, TW, TG;
  DevBuf<double> Cb, A2, Wx;   // eigenbasis CG: P^T R, P^T at2 P, the carried rows for x (see schur_eig)
  DevBuf<double> KK, H0, phia2;   // Kt o Kt (Kt = R^T R); Q/(2 lambda2) + KK/mu; Phi(at2)
  DevBuf<double> CbT;             // Cb^T, for the few-row form of the Schur operator
  DevBuf<double> v1, v2, v3, v4, v5, v6, w1, w2, w3;
  DevBuf<double> Fvg, FvX;     // F(v) of the EG iterate, from its last residual evaluation
  bool fv_valid = false;
  DevBuf<double> Plast;        // most recent non-trivial eigenbasis of the running solve
  bool plast_valid = false, in_solve = false;
  DevBuf<double> partial, scal, bounds;
  DevBuf<int> iscal;
  double* hs = nullptr;                        // pinned host scalars
  int* hi = nullptr;
  JacobiWork jw;
  TcWork tc;
  OzWork oz;              // mixed form: FP64-accurate products emulated on the tensor cores
  bool force64 = false;   // mixed form: run the Newton-direction products in FP64 for now
  long long eig_calls = 0, eig_sweeps = 0, eig_refined = 0, eig_refine_steps = 0;
  DevBuf<double> eZ, eP, esig;   // kot_eig_sym: symmetrised input and outputs
  std::vector<double> hist;
  std::vector<double> trace;   // per iteration: ||R||, mu, CG steps, theta, direction kind
  int last_dir_kind = 0;       // 0 FP64, 1 tensor cores, 2 tensor cores + FP64 refinement
  Profiler prof;
  // Algorithm 2's extragradient sequence v runs beside the Newton step on w (they meet only in
  // the acceptance test): its own context (buffers, stream, workspaces) driven by a helper
  // host thread, so that one sequence's readbacks overlap the other's GPU work.
  kot_ctx* lane = nullptr;
  kot_ctx* owner = nullptr;          // set in the lane: the context whose profiler it shares
  std::thread lane_thread;
  std::mutex lane_mu;
  std::condition_variable lane_cv;
  int lane_job = 0;                  // 0 idle, 1 run one EG step and R(v), 2 quit
  bool lane_busy = false;
  double lane_eta = 0.0;
  std::exception_ptr lane_err;
  cudaEvent_t lane_ev = nullptr;     // this context's reads of the lane's buffers, awaited by the lane
};

namespace {

constexpr int kMaxSweeps = 40;

void set_defaults(kot_options* o) {
  std::memset(o, 0, sizeof(*o));
  o->device = 0;
  o->stream = nullptr;
  o->precision = KOT_FP64;
  o->host_pointers = 0;
  o->max_iter = 200;
  o->cg_max_iter = 20;
  o->tau = 0.1;
  o->kappa = 1.0;
  o->alpha1 = 1e-6;
  o->alpha2 = 1.0;
  o->beta0 = 0.5;
  o->beta1 = 1.2;
  o->beta2 = 5.0;
  o->theta0 = 1.0;
  o->theta_min = 1e-6;
  o->theta_max = 1e6;
  o->eg_step = 0.0;
  o->jitter = 1e-10;
  o->jitter_max = 1e-6;
  o->use_eg = 1;
  o->record_history = 0;
  o->eig_ctas = 0;
  o->mixed_switch = 1e-4;
  o->batch_workers = 0;
  o->eig_refine = 5;
  o->schur_solver = 0;
  o->tc_min_flops = 8e6;
}

bool pos_finite(double v) { return std::isfinite(v) && v > 0.0; }

void fail(kot_status s, const std::string& what) { throw Error{s, what}; }

// ------------------------------------------------------------------ buffers and I/O
void ensure(kot_ctx* C, int l) {
  const size_t L2 = (size_t)l * l, L = (size_t)l;
  for (DevBuf<double>* b : {&C->Q, &C->K, &C->R, &C->X, &C->vX, &C->tX, &C->dX, &C->M1, &C->M2,
                            &C->M3, &C->M4, &C->M5, &C->M6, &C->TU, &C->TV, &C->TW, &C->TG,
                            &C->Cb, &C->A2, &C->Wx, &C->rw.r2, &C->rv.r2, &C->rt.r2, &C->FvX,
                            &C->Plast, &C->KK, &C->H0, &C->CbT})
    b->alloc(L2);
  C->Fvg.alloc(L);
  for (DevBuf<double>* b : {&C->z, &C->w_mu, &C->w_nu, &C->c, &C->g, &C->vg, &C->tg, &C->dg,
                            &C->v1, &C->v2, &C->v3, &C->v4, &C->v5, &C->v6, &C->w1, &C->w2,
                            &C->w3, &C->rw.r1, &C->phia2,
                            &C->rv.r1, &C->rt.r1})
    b->alloc(L);
  for (EigSlot* e : {&C->ew, &C->ev, &C->et, &C->e1, &C->e2}) {
    e->P.alloc(L2);
    e->sig.alloc(L);
  }
  C->partial.alloc(std::max(kReduceBlocks, 64));
  C->scal.alloc(64);
  C->bounds.alloc(2 + 2 * L);
  C->iscal.alloc(16);
}

// Input array -> device pointer (copies host arrays into staging slot k).
const double* dev_in(kot_ctx* C, int k, const double* p, size_t count) {
  if (!C->opt.host_pointers) return p;
  C->stage[k].alloc(count);
  KOT_CUDA(cudaMemcpyAsync(C->stage[k].p, p, count * sizeof(double), cudaMemcpyHostToDevice, C->st));
  return C->stage[k].p;
}

// Copy a device result to the caller's array (device or host).
void dev_out(kot_ctx* C, double* dst, const double* src, size_t count) {
  if (!dst) return;
  KOT_CUDA(cudaMemcpyAsync(dst, src, count * sizeof(double),
                           C->opt.host_pointers ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                           C->st));
}

void fetch(kot_ctx* C, int count) {
  KOT_CUDA(cudaMemcpyAsync(C->hs, C->scal.p, count * sizeof(double), cudaMemcpyDeviceToHost, C->st));
  KOT_CUDA(cudaStreamSynchronize(C->st));
}

// FP64-accurate products of the mixed form run emulated on the tensor cores (gemm_oz); the FP64
// form keeps them on the FP64 pipes.
OzWork* ozp(kot_ctx* C) { return C->opt.precision == KOT_MIXED ? &C->oz : nullptr; }

// ------------------------------------------------------------------ operators (Sec. 4.1)
// out = Phi*(gamma) = R diag(gamma) R^T
void phi_star(kot_ctx* C, const double* gamma, double* out) {
  const int l = C->l;
  gemm_acc(C->st, ozp(C), false, true, l, l, l, 1.0, C->R.p, l, C->R.p, l, gamma, 0.0, out, l,
           G_KLO_ROW | G_KLO_COL | G_SYM);
}

// out = Phi(X)_i = (R^T X R)_ii ; tmp: l x l scratch
void phi(kot_ctx* C, const double* X, double* out, double* tmp) {
  const int l = C->l;
  gemm_acc(C->st, ozp(C), false, false, l, l, l, 1.0, X, l, C->R.p, l, nullptr, 0.0, tmp, l, G_KHI_COL);
  coldot_upper(C->st, l, C->R.p, tmp, out);
}

// ---- the same operators on the tensor cores (mixed form, Newton direction only) ----
bool mixed(const kot_ctx* C) { return C->opt.precision == KOT_MIXED && !C->force64; }
// Slices per operand of the reduced-precision Jacobian products inside CG: three BF16 slices,
// i.e. the six BF16 x BF16 products (FP32 accumulation) of a three-term split, about FP32
// accuracy; the FP64-accuracy products of the mixed form use oz.slices (six).
constexpr int kCgSlices = 3;

void phi_star_nd(kot_ctx* C, const double* gamma, double* out) {
  if (!mixed(C)) return phi_star(C, gamma, out);
  const int l = C->l;
  // out[m][n] = sum_k R[m][k] gamma_k R[n][k]
  gemm_oz(C->st, C->oz, l, l, l, TcOperand{C->R.p, l, false, gamma}, TcOperand{C->R.p, l, false, nullptr},
          kCgSlices, 1.0, 0.0, out, l, true);
}

void phi_nd(kot_ctx* C, const double* X, double* out, double* tmp) {
  if (!mixed(C)) return phi(C, X, out, tmp);
  const int l = C->l;
  // tmp = X R: tmp[m][n] = sum_k X[m][k] R[k][n]
  gemm_oz(C->st, C->oz, l, l, l, TcOperand{X, l, false, nullptr}, TcOperand{C->R.p, l, true, nullptr},
          kCgSlices, 1.0, 0.0, tmp, l, false);
  coldot_upper(C->st, l, C->R.p, tmp, out);
}

// out = (Q gamma - z)/(2 lambda2) - Phi(X)
void grad_gamma(kot_ctx* C, const double* gamma, const double* X, double* out, double* vtmp,
                double* mtmp) {
  const int l = C->l;
  phi(C, X, vtmp, mtmp);
  grad_gamma_fused(C->st, l, 1.0 / (2.0 * C->lambda2), C->Q.p, gamma, C->z.p, vtmp, out);
}

// Eigen-decompose Z (read only) into slot e (warm-started from `warm` if valid); reads the
// alpha-bar count back to the host.
void eig_into(kot_ctx* C, const double* Z, EigSlot& e, const EigSlot* warm) {
  Range range("kot/eig");
  const int l = C->l;
  // Warm start: the previous basis of the same sequence; inside a solve, when that is missing or
  // only the identity of a diagonal matrix (the start, w0 = v0 = 0), the most recent non-trivial
  // basis of any sequence (e.g. R(v1) from the EG projection just computed) -- refinement falls
  // back to Jacobi sweeps when it is too far off.
  const double* wp = (warm && warm->valid && !warm->trivial) ? warm->P.p : nullptr;
  if (!wp && C->in_solve && C->plast_valid) wp = C->Plast.p;
  // Second candidate: the slot's own previous basis.  R(w~) starts from the current iterate's
  // basis; after a rejected Newton step the next trial point lies near the last one, whose basis
  // this slot still holds, so it refines where the iterate's basis is too far off.
  const double* wp2 =
      (C->in_solve && &e != warm && e.valid && !e.trivial && e.P.p != wp) ? e.P.p : nullptr;
  // Mixed form: a refinement whose correction is <= 1e-6 leaves a basis accurate to ~1e-12,
  // below the accuracy of its emulated products; the eigenvalues (Rayleigh quotients, which decide
  // alpha and Omega) are accurate to second order.  The FP64 form refines to FP64 rounding.
  C->jw.refine_done = C->opt.precision == KOT_MIXED ? 1e-6 : 1e-8;
  C->eig_sweeps += eig_sym_f64(C->st, l, Z, wp, e.P.p, e.sig.p, C->jw, kMaxSweeps, C->hs,
                               C->opt.eig_ctas, C->opt.eig_refine, wp2);
  C->eig_calls += 1;
  C->eig_refined += C->jw.last_refine > 0;
  C->eig_refine_steps += C->jw.last_refine;
  if (C->jw.last_nb >= 0) {
    e.nb = C->jw.last_nb;   // counted by the refinement's last step, read with its convergence test
  } else {
    count_nonpos(C->st, l, e.sig.p, C->iscal.p);
    KOT_CUDA(cudaMemcpyAsync(C->hi, C->iscal.p, sizeof(int), cudaMemcpyDeviceToHost, C->st));
    KOT_CUDA(cudaStreamSynchronize(C->st));
    e.nb = C->hi[0];
  }
  e.valid = true;
  e.trivial = wp == nullptr && C->jw.last_trivial;
  if (C->in_solve && !e.trivial) {
    KOT_CUDA(cudaMemcpyAsync(C->Plast.p, e.P.p, (size_t)l * l * sizeof(double), cudaMemcpyDeviceToDevice, C->st));
    C->plast_valid = true;
  }
}

// out = Pi_{S+}(Z) from slot e (Eq. (4.4)); out may alias Z.
void form_proj(kot_ctx* C, const double* Z, const EigSlot& e, double* out) {
  const int l = C->l, nb = e.nb, na = l - nb;
  if (na == 0) {
    fill(C->st, (size_t)l * l, 0.0, out);
  } else if (na <= nb) {
    const double* Pa = e.P.p + nb;
    gemm_acc(C->st, ozp(C), false, true, l, l, na, 1.0, Pa, l, Pa, l, e.sig.p + nb, 0.0, out, l, G_SYM);
  } else {
    // Pi_{S+}(Z) = Z - P_abar diag(sig_abar) P_abar^T (fewer columns)
    if (out != Z) copy_mat(C->st, l, l, Z, l, out, l);
    if (nb > 0)
      gemm_acc(C->st, ozp(C), false, true, l, l, nb, -1.0, e.P.p, l, e.P.p, l, e.sig.p, 1.0, out, l, G_SYM);
  }
}

// out <- Pi_{S+}(sym(X - a S) - c I) with slot e (warm-started from itself); out may alias X.
void proj_into(kot_ctx* C, const double* X, const double* S, double a, double c, double* out, EigSlot& e) {
  const int l = C->l;
  form_z(C->st, l, X, S, a, c, C->M6.p, nullptr);
  eig_into(C, C->M6.p, e, &e);
  form_proj(C, C->M6.p, e, out);
}

// R(w) of Eq. (4.2) into r; eigen-decomposition of Z(w) into e.
// save_fv: (gamma, X) is the EG iterate v; keep F(v) = (r1, Phi*(gamma) + lambda1 I) for the next
// extragradient step, which starts by evaluating exactly these (same kernels, same bits).
// defer: leave |r1|^2, |r2|^2 in scal[0..1] unread (the caller fetches them together with its
// own scalars and calls finish_residual).
void finish_residual(kot_ctx* C, ResState& r) {
  r.n1 = std::sqrt(C->hs[0]);
  r.n2 = std::sqrt(C->hs[1]);
  r.norm = r.n1 + r.n2;
  if (!std::isfinite(r.norm)) fail(KOT_ERR_NONFINITE, "residual is not finite");
}

void residual(kot_ctx* C, const double* gamma, const double* X, EigSlot& e, const EigSlot* warm,
              ResState& r, bool save_fv = false, bool defer = false) {
  Range range("kot/residual");
  const int l = C->l;
  const size_t L2 = (size_t)l * l;
  phi_star(C, gamma, C->M1.p);
  // Z = sym(X - Phi*(gamma)) - lambda1 I into M5; with save_fv, F_X(v) = Phi*(gamma) + lambda1 I
  form_z(C->st, l, X, C->M1.p, 1.0, C->lambda1, C->M5.p, save_fv ? C->FvX.p : nullptr);
  eig_into(C, C->M5.p, e, warm);
  form_proj(C, C->M5.p, e, C->M2.p);
  grad_gamma(C, gamma, X, r.r1.p, C->v1.p, C->M3.p);           // r1
  if (save_fv) {
    KOT_CUDA(cudaMemcpyAsync(C->Fvg.p, r.r1.p, l * sizeof(double), cudaMemcpyDeviceToDevice, C->st));
    C->fv_valid = true;                                       // F_gamma(v) = r1(v)
  }
  // r2 = X - Pi(Z) with |r1|^2 and |r2|^2 in one pass
  sub_norms(C->st, l, r.r1.p, L2, X, C->M2.p, r.r2.p, C->scal.p, C->partial.p);
  if (defer) return;
  fetch(C, 2);
  finish_residual(C, r);
}

// out = T_k[S] (Sec. 4.3) with the eigen-decomposition in e and regularisation mu.
// |alpha| <= |alpha-bar|: G + G^T with U = P_a^T S (8 |alpha| l^2 flops);
// otherwise the complement form S/mu - P((E/mu - Psi) o (P^T S P))P^T (8 |alpha-bar| l^2).
void t_apply(kot_ctx* C, const EigSlot& e, double mu, const double* S, double* out) {
  const int l = C->l, nb = e.nb, na = l - nb;
  const size_t L2 = (size_t)l * l;
  if (na == 0) {
    fill(C->st, L2, 0.0, out);
    return;
  }
  if (nb == 0) {
    axpby(C->st, L2, 1.0 / mu, S, 0.0, nullptr, out);
    return;
  }
  const bool comp = na > nb;
  const int rows = comp ? nb : na;
  const double* Ps = comp ? e.P.p : e.P.p + nb;   // l x rows, ld l
  if (mixed(C)) {
    cudaStream_t st = C->st;
    OzWork& w = C->oz;
    // U = Ps^T S ; V = U P ; weights ; W = V P^T ; G = Ps W   (C = op(A) op(B)^T form)
    gemm_oz(st, w, rows, l, l, TcOperand{Ps, l, true, nullptr}, TcOperand{S, l, true, nullptr}, kCgSlices, 1.0,
            0.0, C->TU.p, l, false);
    gemm_oz(st, w, rows, l, l, TcOperand{C->TU.p, l, false, nullptr}, TcOperand{e.P.p, l, true, nullptr},
            kCgSlices, 1.0, 0.0, C->TV.p, l, false);
    t_weights(st, l, nb, e.sig.p, mu, comp ? 1 : 0, C->TV.p);
    gemm_oz(st, w, rows, l, l, TcOperand{C->TV.p, l, false, nullptr}, TcOperand{e.P.p, l, false, nullptr},
            kCgSlices, 1.0, 0.0, C->TW.p, l, false);
    gemm_oz(st, w, l, l, rows, TcOperand{Ps, l, false, nullptr}, TcOperand{C->TW.p, l, true, nullptr},
            kCgSlices, 1.0, 0.0, C->TG.p, l, false);
  } else {
    gemm_acc(C->st, ozp(C), true, false, rows, l, l, 1.0, Ps, l, S, l, nullptr, 0.0, C->TU.p, l, 0);
    gemm_acc(C->st, ozp(C), false, false, rows, l, l, 1.0, C->TU.p, l, e.P.p, l, nullptr, 0.0, C->TV.p, l, 0);
    t_weights(C->st, l, nb, e.sig.p, mu, comp ? 1 : 0, C->TV.p);
    gemm_acc(C->st, ozp(C), false, true, rows, l, l, 1.0, C->TV.p, l, e.P.p, l, nullptr, 0.0, C->TW.p, l, 0);
    gemm_acc(C->st, ozp(C), false, false, l, l, rows, 1.0, Ps, l, C->TW.p, l, nullptr, 0.0, C->TG.p, l, 0);
  }
  sym_sum(C->st, l, C->TG.p, S, 1.0 / mu, comp ? 1 : 0, out);
}

// The Schur operator of Algorithm 1 in the eigenbasis of Z = P diag(sig) P^T.  With Cb = P^T R
// (row j: eigen-index j, column i: point i), P^T Phi*(p) P = Cb diag(p) Cb^T, so
// T[Phi*(p)] = P (Psi o Cb diag(p) Cb^T) P^T and Phi(T[Phi*(p)]) = diag(Cb^T (Psi o ...) Cb).  Psi
// (Sec. 4.3) is symmetric and vanishes on alpha-bar x alpha-bar, so its alpha rows determine the
// product: with W = the alpha rows of Psi o Cb diag(p) Cb^T, the alpha x alpha block halved (the
// weights of the G + G^T form), T[Phi*(p)] = G + G^T for G = P_alpha W P^T and
// Phi(T[Phi*(p)]) = 2 diag(Cb_alpha^T W Cb).  That is two |alpha| x l x l products per operator
// application, against 2 l^3 + 4 min(|alpha|, |alpha-bar|) l^2 multiply-adds for
// phi_star / T / phi.  Products run at the phase's precision (three slices inside tensor-core CG).
// Out: W (|alpha| x l, ld l), Hp = Q p/(2 lambda2) + mu p + Phi(T[Phi*(p)]); Y: |alpha| x l scratch.
// Products small enough for gemm_acc's FP64 route (OzWork::f64_below) run exact in either phase.
bool cg_products_exact(const kot_ctx* C, int rows) {
  return 2.0 * rows * (double)C->l * C->l < C->oz.f64_below;
}

void cg_gemm(kot_ctx* C, bool ta, bool tb, int M, int N, int K, const double* A, const double* B,
             const double* s, double* out) {
  const int l = C->l;
  if (mixed(C) && 2.0 * M * (double)N * K >= C->oz.f64_below)
    gemm_oz(C->st, C->oz, M, N, K, TcOperand{A, l, ta, s}, TcOperand{B, l, !tb, nullptr}, kCgSlices, 1.0, 0.0,
            out, l, false);
  else
    gemm_acc(C->st, ozp(C), ta, tb, M, N, K, 1.0, A, l, B, l, s, 0.0, out, l, 0);
}

// Complement form (|alpha| > |alpha-bar|, the last paragraph of Sec. 4.3): with Psi' = E/mu - Psi,
// which vanishes on alpha x alpha, Psi o V = V/mu - Psi' o V and, for orthogonal P,
// diag(Cb^T V Cb) = (Kt o Kt) p with Kt = R^T R.  So Phi(T[Phi*(p)]) = (Kt o Kt) p/mu
// - 2 diag(Cb_abar^T W' Cb), W' = the alpha-bar rows U = Cb_abar diag(p) Cb^T weighted by 1/(2 mu)
// on alpha-bar columns and 1/mu - xi on alpha columns: two |alpha-bar| x l x l products plus the
// matvec with H0 = Q/(2 lambda2) + (Kt o Kt)/mu, formed once per direction.  Either way one
// operator application costs 2 min(|alpha|, |alpha-bar|) l^2 multiply-adds in products.
// Out: W = the carried rows for p -- the weighted alpha rows (G + G^T form) or the unweighted
// alpha-bar rows U (complement form) -- and Hp = Q p/(2 lambda2) + mu p + Phi(T[Phi*(p)]);
// Y: rows x l scratch.
bool complement_form(const EigSlot& e, int l) { return l - e.nb > e.nb; }

// Few carried rows (1 .. kSkinnyRows): the FP64 row and column kernels of newton.cu (CbT = Cb^T
// formed once per direction), exact and two launches instead of two products and four launches.
bool skinny_form(const EigSlot& e, int l) {
  const int crow = complement_form(e, l) ? e.nb : l - e.nb;
  return crow > 0 && crow <= kSkinnyRows;
}

void schur_eig(kot_ctx* C, const EigSlot& e, double mu, const double* p, double* W, double* Y, double* Hp) {
  const int l = C->l, nb = e.nb, na = l - nb;
  cudaStream_t st = C->st;
  const double* Cb = C->Cb.p;
  if (skinny_form(e, l)) {
    const bool comp = complement_form(e, l);
    const int crow = comp ? nb : na, r0 = comp ? 0 : nb;
    schur_rows(st, l, crow, r0, Cb, p, e.sig.p, mu, nb, comp ? 1 : 0, W, Y);
    if (comp) schur_cols(st, l, crow, r0, C->CbT.p, Y, -2.0, C->H0.p, 1.0, p, mu, Hp);
    else schur_cols(st, l, crow, r0, C->CbT.p, Y, 2.0, C->Q.p, 1.0 / (2.0 * C->lambda2), p, mu, Hp);
    return;
  }
  if (complement_form(e, l)) {
    if (nb == 0) {
      fill(st, l, 0.0, C->v5.p);
    } else {
      cg_gemm(C, false, true, nb, l, l, Cb, Cb, p, W);       // U = Cb_abar diag(p) Cb^T
      t_weights(st, l, nb, e.sig.p, mu, 1, Y, W);            // W' = weights o U
      cg_gemm(C, false, false, nb, l, l, Y, Cb, nullptr, C->TU.p);   // W' Cb
      coldot_rows(st, nb, l, Cb, l, C->TU.p, l, -2.0, C->v5.p);
    }
    hmatvec(st, l, 1.0, C->H0.p, p, mu, C->v5.p, Hp);
    return;
  }
  const double* Ca = Cb + (size_t)nb * l;
  if (na == 0) {
    fill(st, l, 0.0, C->v5.p);
  } else {
    cg_gemm(C, false, true, na, l, l, Ca, Cb, p, W);     // W = Cb_alpha diag(p) Cb^T
    t_weights(st, l, nb, e.sig.p, mu, 0, W);
    cg_gemm(C, false, false, na, l, l, W, Cb, nullptr, Y);   // Y = W Cb
    coldot_rows(st, na, l, Ca, l, Y, l, 2.0, C->v5.p);
  }
  hmatvec(st, l, 1.0 / (2.0 * C->lambda2), C->Q.p, p, mu, C->v5.p, Hp);
}

// Symmetric QMR (Freund and Nachtigal, no preconditioner) on H x = a1 from the x in dgam, whose
// residual a1 - H x is in ev and T[Phi*(x)] in TPx.  The Lanczos residual rl drives the
// recurrences; x moves along the smoothed direction d, and the true residual and T[Phi*(x)]
// follow through H d and T[Phi*(d)], so the stopping test of Eq. (4.3) (or cg_tol_abs) sees the
// returned iterate's own residual.  Returns the iterations; met = whether the test held.
int sqmr_loop(kot_ctx* C, const ResState& r, const EigSlot& e, double mu, double cg_tol_abs, int cap,
              const double* at2, const double* a1, double* dgam, double* TPx, double* ev, bool& met) {
  (void)a1;
  const int l = C->l;
  const size_t L2 = (size_t)l * l;
  cudaStream_t st = C->st;
  double* rl = C->w1.p;      // Lanczos residual
  double* q = C->v4.p;       // direction of the recurrences
  double* t = C->v6.p;       // H q
  double* d = C->w2.p;       // iterate update
  double* Hd = C->w3.p;      // H d
  double* TPd = C->M2.p;     // T[Phi*(d)]  (M2 is free once the right-hand side is formed)
  KOT_CUDA(cudaMemcpyAsync(rl, ev, l * sizeof(double), cudaMemcpyDeviceToDevice, st));
  KOT_CUDA(cudaMemcpyAsync(q, ev, l * sizeof(double), cudaMemcpyDeviceToDevice, st));
  fill(st, l, 0.0, d);
  fill(st, l, 0.0, Hd);
  fill(st, L2, 0.0, TPd);
  sumsq_f64(st, l, rl, C->scal.p, C->partial.p);
  fetch(C, 1);
  double rho = C->hs[0], tau_q = std::sqrt(rho), theta = 0.0;
  int it = 0;
  while (true) {
    two_norms(st, l, dgam, L2, at2, TPx, C->scal.p + 1, C->partial.p);
    sumsq_f64(st, l, ev, C->scal.p, C->partial.p);
    fetch(C, 3);
    const double enorm = std::sqrt(C->hs[0]);
    if (!std::isfinite(enorm)) fail(KOT_ERR_NONFINITE, "QMR residual is not finite");
    bool stop;
    if (cg_tol_abs > 0) stop = enorm <= cg_tol_abs;
    else {
      const double dw = std::sqrt(C->hs[1]) + std::sqrt(C->hs[2]);
      stop = enorm <= C->opt.tau * std::min(1.0, C->opt.kappa * r.norm * dw);
    }
    met = stop;
    if (stop || it >= cap) break;
    // t = H q, M6 = T[Phi*(q)]
    phi_star_nd(C, q, C->M5.p);
    t_apply(C, e, mu, C->M5.p, C->M6.p);
    phi_nd(C, C->M6.p, C->v5.p, C->M5.p);
    hmatvec(st, l, 1.0 / (2.0 * C->lambda2), C->Q.p, q, mu, C->v5.p, t);
    dot_f64(st, l, q, t, C->scal.p + 3, C->partial.p);
    fetch(C, 4);
    const double sig = C->hs[3];
    if (!(sig > 0.0) || tau_q == 0.0) break;
    const double a = rho / sig;
    axpby(st, l, 1.0, rl, -a, t, rl);
    sumsq_f64(st, l, rl, C->scal.p + 4, C->partial.p);
    KOT_CUDA(cudaMemcpyAsync(C->hs + 4, C->scal.p + 4, sizeof(double), cudaMemcpyDeviceToHost, st));
    KOT_CUDA(cudaStreamSynchronize(st));
    const double rr = C->hs[4];
    const double theta_old = theta;
    theta = std::sqrt(rr) / tau_q;
    const double c2 = 1.0 / (1.0 + theta * theta);
    tau_q = tau_q * theta * std::sqrt(c2);
    const double f = c2 * theta_old * theta_old, g = c2 * a;
    axpby(st, l, f, d, g, q, d);
    axpby(st, l, f, Hd, g, t, Hd);
    axpby(st, L2, f, TPd, g, C->M6.p, TPd);
    axpby(st, l, 1.0, dgam, 1.0, d, dgam);
    axpby(st, L2, 1.0, TPx, 1.0, TPd, TPx);
    axpby(st, l, 1.0, ev, -1.0, Hd, ev);
    const double rho_old = rho;
    rho = rr;
    axpby(st, l, 1.0, rl, rho / rho_old, q, q);
    ++it;
  }
  return it;
}

// Algorithm 1 at w (residual r, eigen-decomposition e).  Returns CG iterations.
// Mixed form: CG runs with tensor-core products first.  Its recursive residual belongs to the
// inexact operator, so the test of Eq. (4.3) is then re-taken in FP64: the right-hand side is
// recomputed, the true residual a1 - H x of the mixed solution is formed, and CG continues from
// that x with FP64 products (up to cg_max_iter more iterations) until the FP64 test holds.  The
// returned direction therefore meets Eq. (4.3) as FP64 measures it; without this check the
// directions' ~1e-7/mu error makes rho_k small once mu_k = theta_k ||r_k|| is small, the theta
// rule multiplies theta by beta2, and convergence turns linear.
int newton_direction(kot_ctx* C, const ResState& r, const EigSlot& e, double mu, double cg_tol_abs,
                     double* dgam, double* dX, bool allow_tc) {
  Range range("kot/newton_direction");
  const int l = C->l;
  C->force64 = !allow_tc;
  const size_t L2 = (size_t)l * l;
  cudaStream_t st = C->st;
  double* rT = C->M1.p;     // r2 + T[r2]
  double* at2 = C->M3.p;    // (a2 + T[a2])/(mu + 1)
  double* TPx = C->M4.p;    // T[Phi*(x)]
  double* a1 = C->v2.p;
  double* ev = C->v3.p;     // CG residual
  double* pv = C->v4.p;     // CG direction
  double* Hp = C->v6.p;
  const int cap = cg_tol_abs > 0 ? 10 * l + 50 : C->opt.cg_max_iter;
  // the few-row form of the operator, and products small enough for the FP64 GEMM, run in FP64
  // in both forms, so their directions need no FP64 re-check
  const bool skinny = C->opt.schur_solver != 1 && skinny_form(e, l);
  const int nb0 = e.nb, crow0 = complement_form(e, l) ? nb0 : l - nb0;
  const bool exact_ops = skinny || (C->opt.schur_solver != 1 && cg_products_exact(C, crow0));
  const bool refine = mixed(C) && !exact_ops;
  int total = 0, refined_steps = 0;
  bool met = false;
  // right-hand side: a1 = -r1 - Phi(r2 + T[r2])/(mu+1), at2 = -(r2 + T[r2])/(mu+1), formed
  // once with FP64-accuracy products (CG iterates, not the system, carry the reduced precision).
  // CG works on the eigenbasis form of the operator (see schur_eig) and forms the right-hand
  // side there too: with Cb = P^T R and B = P^T r2 P, A2 = P^T at2 P = -(1 + Psi) o B/(mu + 1)
  // and Phi(at2) = diag(Cb^T A2 Cb), so a1 = -r1 + diag(Cb^T A2 Cb); the stopping test reads A2
  // (and |A2 on alpha-bar x alpha-bar|^2), and the direction ends as dX = P (A2 - P^T T[Phi*(x)] P) P^T.
  // Symmetric QMR keeps the direct form phi_star / T / phi.
  const bool eigcg = C->opt.schur_solver != 1;
  const int nb = e.nb, na = l - nb;
  const bool comp = eigcg && complement_form(e, l);
  const int crow = comp ? nb : na;   // rows carried for T[Phi*(x)] (see schur_eig)
  double* sc = C->scal.p;
  double* Wx = C->Wx.p;
  if (eigcg) {
    OzWork* oz = ozp(C);
    gemm_acc(st, oz, true, false, l, l, l, 1.0, e.P.p, l, C->R.p, l, nullptr, 0.0, C->Cb.p, l, G_KHI_COL);
    if (skinny) transpose(st, l, C->Cb.p, C->CbT.p);
    gemm_acc(st, oz, true, false, l, l, l, 1.0, e.P.p, l, r.r2.p, l, nullptr, 0.0, C->TU.p, l, 0);
    gemm_acc(st, oz, false, false, l, l, l, 1.0, C->TU.p, l, e.P.p, l, nullptr, 0.0, C->TV.p, l, G_SYM);
    rhs_weights(st, l, nb, e.sig.p, mu, C->TV.p, C->A2.p);
    gemm_acc(st, oz, false, false, l, l, l, 1.0, C->A2.p, l, C->Cb.p, l, nullptr, 0.0, C->TW.p, l, 0);
    coldot_rows(st, l, l, C->Cb.p, l, C->TW.p, l, 1.0, C->phia2.p);   // Phi(at2)
    axpby(st, l, -1.0, r.r1.p, 1.0, C->phia2.p, a1);
    if (comp) {
      axpby(st, L2, 1.0 / (2.0 * C->lambda2), C->Q.p, 1.0 / mu, C->KK.p, C->H0.p);
      if (cg_tol_abs <= 0) sumsq_f64(st, L2, C->A2.p, sc + 11, C->partial.p);   // ||A2||^2
    } else if (cg_tol_abs <= 0) {
      eig_norms(st, 0, nullptr, nb, nb, l, 0, C->A2.p, nullptr, nullptr, sc + 10, C->partial.p);
    }
  } else {
    C->force64 = true;
    t_apply(C, e, mu, r.r2.p, rT);
    axpby(st, L2, 1.0, r.r2.p, 1.0, rT, rT);
    phi_nd(C, rT, C->v1.p, C->M2.p);
    axpby(st, l, -1.0, r.r1.p, -1.0 / (mu + 1.0), C->v1.p, a1);
    axpby(st, L2, -1.0 / (mu + 1.0), rT, 0.0, nullptr, at2);
  }
  C->force64 = !allow_tc;
  for (int phase = 0; phase < (refine ? 2 : 1); ++phase) {
    if (phase == 1) C->force64 = true;   // always verify a tensor-core direction in FP64
    if (phase == 0) {
      fill(st, l, 0.0, dgam);
      if (eigcg) fill(st, (size_t)crow * l, 0.0, Wx);
      else fill(st, L2, 0.0, TPx);
      KOT_CUDA(cudaMemcpyAsync(ev, a1, l * sizeof(double), cudaMemcpyDeviceToDevice, st));
    } else {
      // e = a1 - H x with FP64 products, and T[Phi*(x)] recomputed alongside
      if (eigcg) {
        schur_eig(C, e, mu, dgam, Wx, C->M6.p, Hp);
      } else {
        phi_star_nd(C, dgam, C->M5.p);
        t_apply(C, e, mu, C->M5.p, TPx);
        phi_nd(C, TPx, C->v5.p, C->M5.p);
        hmatvec(st, l, 1.0 / (2.0 * C->lambda2), C->Q.p, dgam, mu, C->v5.p, Hp);
      }
      axpby(st, l, 1.0, a1, -1.0, Hp, ev);
    }
    KOT_CUDA(cudaMemcpyAsync(pv, ev, l * sizeof(double), cudaMemcpyDeviceToDevice, st));
    int it = 0;
    if (C->opt.schur_solver == 1) {
      it = sqmr_loop(C, r, e, mu, cg_tol_abs, cap, at2, a1, dgam, TPx, ev, met);
    } else {
      // CG with its step lengths kept on the device: ||e||^2 alternates between scal[5] and
      // scal[6], p^T H p is scal[3], scal[7] flags a non-positive curvature; the host reads the
      // norms of the stopping test (and the flag) once per iteration.  T[Phi*(x)] is carried as
      // the alpha rows Wx of its eigenbasis form, and ||at2 - T[Phi*(x)]||_F is measured there.
      int cur = 0;
      fill(st, 1, 0.0, sc + 7);
      sumsq_f64(st, l, ev, sc + 5, C->partial.p);
      while (true) {
        // stop test at the current iterate: ||e|| vs tau min(1, kappa ||r|| ||dw||)
        if (cg_tol_abs > 0) sumsq_f64(st, l, dgam, sc + 1, C->partial.p);
        else if (comp)
          eig_norms_comp(st, l, dgam, nb, e.sig.p, mu, C->A2.p, Wx, C->KK.p, C->phia2.p, sc + 11, sc + 1,
                         C->partial.p);
        else eig_norms(st, l, dgam, na, l, l, nb, C->A2.p + (size_t)nb * l, Wx, sc + 11, sc + 1, C->partial.p);
        fetch(C, 8);
        const double ee = C->hs[5 + cur];
        const double enorm = std::sqrt(ee);
        if (!std::isfinite(enorm)) {
          C->force64 = false;
          fail(KOT_ERR_NONFINITE, "CG residual is not finite");
        }
        bool stop;
        if (cg_tol_abs > 0) stop = enorm <= cg_tol_abs;
        else {
          const double dw = std::sqrt(C->hs[1]) + std::sqrt(std::max(C->hs[2], 0.0));
          stop = enorm <= C->opt.tau * std::min(1.0, C->opt.kappa * r.norm * dw);
        }
        met = stop;
        if (C->hs[7] != 0.0) {   // the last step met p^T H p <= 0 and was not taken
          --it;
          break;
        }
        if (stop || it >= cap) break;
        // Hp = Q p/(2 lambda2) + mu p + Phi(T[Phi*(p)]); M5 = alpha rows of T[Phi*(p)] (eigenbasis)
        {
          const double L = l, a = std::min(na, nb);
          ProfScope ps(st, KC_MATVEC, 4.0 / 3.0 * L * L * L + 8.0 * a * L * L + 2.0 * L * L,
                       8.0 * (2.0 * L * L + 4.0 * a * L), 4.0 * a * L * L + 2.0 * L * L);
          schur_eig(C, e, mu, pv, C->M5.p, C->M6.p, Hp);
        }
        // a = ||e||^2 / p^T H p: x += a p, e -= a H p, p = e + b p, and the carried rows of
        // T[Phi*(x)] += a those of T[Phi*(p)] (one block, scalars on the device)
        cg_step(st, l, Hp, pv, dgam, ev, sc, cur, (size_t)crow * l, C->M5.p, Wx);
        cur ^= 1;
        ++it;
      }
    }
    total += it;
    if (phase == 1) refined_steps = it;
  }
  // 1: tensor-core direction accepted by the FP64 check as is; 2: FP64 steps were added
  C->last_dir_kind = refine ? (refined_steps == 0 ? 1 : 2) : 0;
  C->force64 = false;
  if (eigcg) {
    // dX = at2 - T[Phi*(x)] = P D P^T, D = A2 - P^T T[Phi*(x)] P (FP64-accuracy products); the
    // complement form carries no alpha rows, so D = A2 - Psi o Vx from Vx = Cb diag(x) Cb^T
    if (comp) {
      gemm_acc(st, ozp(C), false, true, l, l, l, 1.0, C->Cb.p, l, C->Cb.p, l, dgam, 0.0, C->TV.p, l, G_SYM);
      assemble_psi(st, l, nb, e.sig.p, mu, C->A2.p, C->TV.p, C->TG.p);
    } else {
      assemble_dir(st, l, nb, C->A2.p, Wx, C->TG.p);
    }
    gemm_acc(st, ozp(C), false, true, l, l, l, 1.0, C->TG.p, l, e.P.p, l, nullptr, 0.0, C->TW.p, l, 0);
    gemm_acc(st, ozp(C), false, false, l, l, l, 1.0, e.P.p, l, C->TW.p, l, nullptr, 0.0, dX, l, G_SYM);
  } else {
    axpby(st, L2, 1.0, at2, -1.0, TPx, dX);
  }
  return total;   // a timed-out tensor-core wait is reported when the API call returns (run())
}

// One projected extragradient step on (vg, vX) with step eta (Korpelevich).
void eg_step(kot_ctx* C, double eta) {
  Range range("kot/eg_step");
  const int l = C->l;
  const size_t L2 = (size_t)l * l;
  cudaStream_t st = C->st;
  // F at v (kept from the residual of v when that was the last thing computed at v)
  const double* FX = C->M1.p;
  if (C->fv_valid) {
    KOT_CUDA(cudaMemcpyAsync(C->v2.p, C->Fvg.p, l * sizeof(double), cudaMemcpyDeviceToDevice, st));
    FX = C->FvX.p;
  } else {
    grad_gamma(C, C->vg.p, C->vX.p, C->v2.p, C->v1.p, C->M3.p);  // v2 = F_gamma(v)
    phi_star(C, C->vg.p, C->M1.p);
    add_diag(st, l, C->lambda1, C->M1.p, l);                      // M1 = F_X(v)
  }
  axpby(st, l, 1.0, C->vg.p, -eta, C->v2.p, C->v4.p);             // gamma_h
  proj_into(C, C->vX.p, FX, eta, 0.0, C->M2.p, C->e1);            // X_h = Pi(X_v - eta F_X(v))
  // F at h
  grad_gamma(C, C->v4.p, C->M2.p, C->v3.p, C->v1.p, C->M3.p);
  phi_star(C, C->v4.p, C->M1.p);                                  // F_X(h) = M1 + lambda1 I
  axpby(st, l, 1.0, C->vg.p, -eta, C->v3.p, C->vg.p);
  proj_into(C, C->vX.p, C->M1.p, eta, eta * C->lambda1, C->vX.p, C->e2);
  C->fv_valid = false;                                            // v has moved
}

// <R(w~), dw> into scal[2] + scal[3] and |dg|^2, |dX|^2 into scal[4], scal[5] (read with the
// deferred residual of w~ in one fetch)
void pair_inner(kot_ctx* C, const ResState& r, const double* dg, const double* dX) {
  const int l = C->l;
  dot_f64(C->st, l, r.r1.p, dg, C->scal.p + 2, C->partial.p);
  dot_f64(C->st, l * l, r.r2.p, dX, C->scal.p + 3, C->partial.p);
  sumsq_f64(C->st, l, dg, C->scal.p + 4, C->partial.p);
  sumsq_f64(C->st, (size_t)l * l, dX, C->scal.p + 5, C->partial.p);
}

void swap_slots(EigSlot& a, EigSlot& b) {
  std::swap(a.P, b.P);
  std::swap(a.sig, b.sig);
  std::swap(a.nb, b.nb);
  std::swap(a.valid, b.valid);
  std::swap(a.trivial, b.trivial);
}
void swap_res(ResState& a, ResState& b) {
  std::swap(a.r1, b.r1);
  std::swap(a.r2, b.r2);
  std::swap(a.n1, b.n1);
  std::swap(a.n2, b.n2);
  std::swap(a.norm, b.norm);
}

double objective_and_ot(kot_ctx* C, const double* gamma, double* ot) {
  const int l = C->l;
  gemv_f64(C->st, l, 1.0, C->Q.p, gamma, 0.0, C->v1.p);
  dot_f64(C->st, l, gamma, C->v1.p, C->scal.p, C->partial.p);
  dot_f64(C->st, l, gamma, C->z.p, C->scal.p + 1, C->partial.p);
  axpby(C->st, l, 1.0, C->w_mu.p, 1.0, C->w_nu.p, C->v2.p);
  dot_f64(C->st, l, gamma, C->v2.p, C->scal.p + 2, C->partial.p);
  fetch(C, 3);
  const double l2 = C->lambda2;
  *ot = C->q2 / (2 * l2) - C->hs[2] / (2 * l2);
  return C->hs[0] / (4 * l2) - C->hs[1] / (2 * l2) + C->q2 / (4 * l2);
}

void compute_eg_L(kot_ctx* C) {
  const int l = C->l;
  // Kt = R^T R into M1
  gemm_acc(C->st, ozp(C), true, false, l, l, l, 1.0, C->R.p, l, C->R.p, l, nullptr, 0.0, C->M1.p, l,
           G_KHI_ROW | G_KHI_COL | G_SYM);
  rowsum_bounds(C->st, l, C->Q.p, C->M1.p, C->bounds.p);
  square_elems(C->st, (size_t)l * l, C->M1.p, C->KK.p);   // Kt o Kt (complement form of CG)
  KOT_CUDA(cudaMemcpyAsync(C->hs, C->bounds.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, C->st));
  KOT_CUDA(cudaStreamSynchronize(C->st));
  C->eg_L = C->hs[0] / (2 * C->lambda2) + std::sqrt(C->hs[1]);
}

void factor(kot_ctx* C) {
  const int l = C->l;
  k_maxdiag<<<1, 256, 0, C->st>>>(l, C->K.p, C->scal.p);
  KOT_CHECK_LAUNCH();
  fetch(C, 1);
  const double scale = C->hs[0];
  double rel = C->opt.jitter;
  while (true) {
    C->eps = rel * scale;
    copy_mat(C->st, l, l, C->K.p, l, C->R.p, l);
    cholesky_upper_f64(C->st, l, C->R.p, C->eps, C->iscal.p);
    KOT_CUDA(cudaMemcpyAsync(C->hi, C->iscal.p, sizeof(int), cudaMemcpyDeviceToHost, C->st));
    KOT_CUDA(cudaStreamSynchronize(C->st));
    if (C->hi[0] == 0) break;
    rel *= 10.0;
    if (!(rel > 0.0) || rel > C->opt.jitter_max * (1 + 1e-12))
      fail(KOT_ERR_NOT_PD, "K + eps I is not positive definite up to the jitter limit");
  }
}

void reset_slots(kot_ctx* C) {
  for (EigSlot* e : {&C->ew, &C->ev, &C->et, &C->e1, &C->e2}) e->valid = e->trivial = false;
  C->fv_valid = false;
  C->plast_valid = false;
}

// ------------------------------------------------------------------ the EG lane
// The helper thread of a lane context L (L->owner = the solving context O): waits for a job, runs
// one extragradient step on L's iterate v and evaluates R(v) (its last readback leaves L's
// stream idle), reports completion or the error.
void lane_work(kot_ctx* L) {
  kot_ctx* O = L->owner;
  for (;;) {
    double eta = 0.0;
    {
      std::unique_lock<std::mutex> lk(O->lane_mu);
      O->lane_cv.wait(lk, [&] { return O->lane_job != 0; });
      if (O->lane_job == 2) return;
      eta = O->lane_eta;
    }
    std::exception_ptr err;
    try {
      KOT_CUDA(cudaSetDevice(L->opt.device));
      set_current_profiler(O->prof.mask ? &O->prof : nullptr);
      KOT_CUDA(cudaStreamWaitEvent(L->st, O->lane_ev, 0));   // O's copies out of L's buffers
      eg_step(L, eta);
      residual(L, L->vg.p, L->vX.p, L->ev, &L->ev, L->rv, true);
    } catch (...) {
      err = std::current_exception();
    }
    set_current_profiler(nullptr);
    {
      std::lock_guard<std::mutex> lk(O->lane_mu);
      O->lane_err = err;
      O->lane_job = 0;
      O->lane_busy = false;
    }
    O->lane_cv.notify_all();
  }
}

void lane_start(kot_ctx* C, double eta) {
  {
    std::lock_guard<std::mutex> lk(C->lane_mu);
    C->lane_eta = eta;
    C->lane_err = nullptr;
    C->lane_busy = true;
    C->lane_job = 1;
  }
  C->lane_cv.notify_all();
}

// Wait for the lane's step; rethrow its error.
void lane_wait(kot_ctx* C) {
  std::unique_lock<std::mutex> lk(C->lane_mu);
  C->lane_cv.wait(lk, [&] { return !C->lane_busy; });
  std::exception_ptr e = C->lane_err;
  C->lane_err = nullptr;
  lk.unlock();
  if (e) std::rethrow_exception(e);
}

// Leaves no lane step running when the solving thread unwinds.
struct LaneJoin {
  kot_ctx* C = nullptr;
  ~LaneJoin() {
    if (!C) return;
    std::unique_lock<std::mutex> lk(C->lane_mu);
    C->lane_cv.wait(lk, [&] { return !C->lane_busy; });
    C->lane_err = nullptr;
  }
};

// The lane context of C (created on first use: own stream, pinned scalars, helper thread), set up
// for the current features: R, Q, z copied in, iterate v = w, slots and counters reset.
kot_ctx* lane_for_solve(kot_ctx* C) {
  if (!C->lane) {
    kot_ctx* L = new kot_ctx();
    L->opt = C->opt;
    L->opt.stream = nullptr;
    L->owner = C;
    try {
      KOT_CUDA(cudaStreamCreateWithFlags(&L->st, cudaStreamNonBlocking));
      L->own_stream = true;
      KOT_CUDA(cudaMallocHost(&L->hs, 64 * sizeof(double)));
      KOT_CUDA(cudaMallocHost(&L->hi, 16 * sizeof(int)));
      if (!C->lane_ev) KOT_CUDA(cudaEventCreateWithFlags(&C->lane_ev, cudaEventDisableTiming));
    } catch (...) {
      kot_destroy(L);
      throw;
    }
    C->lane = L;
    C->lane_thread = std::thread(lane_work, L);
  }
  kot_ctx* L = C->lane;
  const int l = C->l;
  const size_t L2 = (size_t)l * l;
  L->l = l;
  ensure(L, l);
  L->lambda1 = C->lambda1;
  L->lambda2 = C->lambda2;
  L->jw.oz = L->opt.precision == KOT_MIXED ? &L->oz : nullptr;
  L->oz.f64_below = L->opt.tc_min_flops;
  L->force64 = false;
  reset_slots(L);
  L->in_solve = true;
  L->eig_calls = L->eig_sweeps = L->eig_refined = L->eig_refine_steps = 0;
  cudaStream_t st = C->st;
  KOT_CUDA(cudaMemcpyAsync(L->R.p, C->R.p, L2 * sizeof(double), cudaMemcpyDeviceToDevice, st));
  KOT_CUDA(cudaMemcpyAsync(L->Q.p, C->Q.p, L2 * sizeof(double), cudaMemcpyDeviceToDevice, st));
  KOT_CUDA(cudaMemcpyAsync(L->z.p, C->z.p, l * sizeof(double), cudaMemcpyDeviceToDevice, st));
  KOT_CUDA(cudaMemcpyAsync(L->vg.p, C->g.p, l * sizeof(double), cudaMemcpyDeviceToDevice, st));
  KOT_CUDA(cudaMemcpyAsync(L->vX.p, C->X.p, L2 * sizeof(double), cudaMemcpyDeviceToDevice, st));
  KOT_CUDA(cudaEventRecord(C->lane_ev, st));
  return L;
}

}  // namespace

// ================================================================== C ABI

namespace {
kot_status run(kot_ctx* C, const std::function<void()>& body) {
  struct Install {
    explicit Install(kot_ctx* c) { set_current_profiler(c && c->prof.mask ? &c->prof : nullptr); }
    ~Install() { set_current_profiler(nullptr); }
  } install(C);
  if (C) {
    C->force64 = false;
    C->in_solve = false;
    C->jw.oz = C->opt.precision == KOT_MIXED ? &C->oz : nullptr;
    C->oz.f64_below = C->opt.tc_min_flops;
  }
  try {
    body();
    if (C && C->opt.precision == KOT_MIXED && gemm_oz_error(C->st, C->oz))
      fail(KOT_ERR_TIMEOUT, "tensor-core FP64-emulation wait timed out");
    if (C && C->lane && C->opt.precision == KOT_MIXED && gemm_oz_error(C->lane->st, C->lane->oz))
      fail(KOT_ERR_TIMEOUT, "tensor-core FP64-emulation wait timed out");
    return KOT_OK;
  } catch (const Error& e) {
    if (C) C->err = e.what;
    return e.status;
  } catch (const std::exception& e) {
    if (C) C->err = e.what();
    return KOT_ERR_CUDA;
  }
}
}  // namespace

extern "C" {

kot_status kot_default_options(kot_options* opt) {
  if (!opt) return KOT_ERR_INVALID;
  set_defaults(opt);
  return KOT_OK;
}

kot_status kot_create(kot_ctx** out, const kot_options* opt) {
  if (!out) return KOT_ERR_INVALID;
  *out = nullptr;
  kot_options o;
  if (opt) o = *opt;
  else set_defaults(&o);
  if (o.max_iter < 0 || o.cg_max_iter < 0 || !(o.tau > 0 && o.tau < 1) || !(o.kappa > 0) ||
      !(o.alpha1 > 0) || !(o.alpha2 >= o.alpha1) || !(o.beta0 > 0) || !(o.beta1 > 0) ||
      !(o.beta2 > 0) || !(o.theta0 > 0) || !(o.theta_min > 0) || !(o.theta_max >= o.theta_min) ||
      !(o.jitter >= 0) || !(o.jitter_max >= o.jitter) || o.eig_ctas < 0 || !(o.mixed_switch >= 0) || o.batch_workers < 0 || o.eig_refine < 0 ||
      (o.schur_solver != 0 && o.schur_solver != 1) || (o.gram_fp32 != 0 && o.gram_fp32 != 1) ||
      !(o.tc_min_flops >= 0 && std::isfinite(o.tc_min_flops)) ||
      (o.precision != KOT_FP64 && o.precision != KOT_MIXED))
    return KOT_ERR_INVALID;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || o.device < 0 || o.device >= ndev) {
    cudaGetLastError();
    return KOT_ERR_CUDA;
  }
  kot_ctx* C = new kot_ctx();
  C->opt = o;
  kot_status s = run(C, [&] {
    KOT_CUDA(cudaSetDevice(o.device));
    if (o.stream) {
      C->st = (cudaStream_t)o.stream;
    } else {
      KOT_CUDA(cudaStreamCreateWithFlags(&C->st, cudaStreamNonBlocking));
      C->own_stream = true;
    }
    KOT_CUDA(cudaMallocHost(&C->hs, 64 * sizeof(double)));
    KOT_CUDA(cudaMallocHost(&C->hi, 16 * sizeof(int)));
  });
  if (s != KOT_OK) {
    kot_destroy(C);
    return s;
  }
  *out = C;
  return KOT_OK;
}

kot_status kot_destroy(kot_ctx* C) {
  if (!C) return KOT_OK;
  cudaSetDevice(C->opt.device);
  if (C->lane) {
    {
      std::lock_guard<std::mutex> lk(C->lane_mu);
      C->lane_job = 2;
    }
    C->lane_cv.notify_all();
    if (C->lane_thread.joinable()) C->lane_thread.join();
    kot_destroy(C->lane);
    C->lane = nullptr;
  }
  if (C->lane_ev) cudaEventDestroy(C->lane_ev);
  if (C->st) cudaStreamSynchronize(C->st);
  for (DevBuf<double>* b : {&C->Q, &C->K, &C->R, &C->z, &C->w_mu, &C->w_nu, &C->c, &C->g, &C->X,
                            &C->vg, &C->vX, &C->tg, &C->tX, &C->dg, &C->dX, &C->M1, &C->M2,
                            &C->M3, &C->M4, &C->M5, &C->M6, &C->TU, &C->TV, &C->TW, &C->TG,
                            &C->Cb, &C->A2, &C->Wx, &C->KK, &C->H0, &C->phia2, &C->CbT,
                            &C->v1, &C->v2, &C->v3, &C->v4, &C->v5, &C->v6, &C->w1, &C->w2,
                            &C->w3, &C->partial,
                            &C->scal, &C->bounds, &C->rw.r1, &C->rw.r2, &C->rv.r1, &C->rv.r2,
                            &C->rt.r1, &C->rt.r2, &C->eZ, &C->eP, &C->esig, &C->sX, &C->sY,
                            &C->sXf, &C->sYf, &C->Fvg, &C->FvX, &C->Plast})
    b->release();
  C->jw.release();
  C->tc.a.release();
  C->tc.b.release();
  C->tc.err.release();
  C->oz.release();
  for (auto& b : C->stage) b.release();
  for (EigSlot* e : {&C->ew, &C->ev, &C->et, &C->e1, &C->e2}) {
    e->P.release();
    e->sig.release();
  }
  C->iscal.release();
  if (C->hs) cudaFreeHost(C->hs);
  if (C->hi) cudaFreeHost(C->hi);
  C->prof.release();
  if (C->own_stream && C->st) cudaStreamDestroy(C->st);
  delete C;
  return KOT_OK;
}

const char* kot_last_error(const kot_ctx* C) { return C ? C->err.c_str() : "null context"; }

kot_status kot_build_features(kot_ctx* C, int d, int n, const double* X, const double* Y, int l,
                              const double* Xf, const double* Yf, double sigma, double lambda1,
                              double lambda2) {
  if (!C) return KOT_ERR_INVALID;
  if (d < 1 || n < 1 || l < 1 || d > 65536 || l > 32768 || !X || !Y || !Xf || !Yf ||
      !pos_finite(sigma) || !pos_finite(lambda1) || !pos_finite(lambda2)) {
    C->err = "kot_build_features: invalid argument";
    return KOT_ERR_INVALID;
  }
  return run(C, [&] {
    Range range("kot/build_features");
    KOT_CUDA(cudaSetDevice(C->opt.device));
    C->have = false;
    C->have_samples = false;
    C->l = l;
    ensure(C, l);
    reset_slots(C);
    cudaStream_t st = C->st;
    const double* dX = dev_in(C, 0, X, (size_t)n * d);
    const double* dY = dev_in(C, 1, Y, (size_t)n * d);
    const double* dXf = dev_in(C, 2, Xf, (size_t)l * d);
    const double* dYf = dev_in(C, 3, Yf, (size_t)l * d);
    const double inv2s2 = 1.0 / (2.0 * sigma * sigma);
    embed_f64(st, n, d, l, dX, dXf, inv2s2, C->w_mu.p);
    embed_f64(st, n, d, l, dY, dYf, inv2s2, C->w_nu.p);
    const int pb = pair_blocks(n);
    C->stage[7].alloc(pb);
    pair_mean_f64(st, n, d, dX, inv2s2, C->scal.p + 10, C->stage[7].p, pb);
    pair_mean_f64(st, n, d, dY, inv2s2, C->scal.p + 11, C->stage[7].p, pb);
    gram_f64(st, l, d, dXf, dYf, inv2s2, lambda2, C->w_mu.p, C->w_nu.p, C->Q.p, C->K.p, C->c.p, C->z.p,
             C->opt.gram_fp32 != 0);
    KOT_CUDA(cudaMemcpyAsync(C->hs + 10, C->scal.p + 10, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    KOT_CUDA(cudaStreamSynchronize(st));
    C->q2 = C->hs[10] + C->hs[11];
    C->lambda1 = lambda1;
    C->lambda2 = lambda2;
    factor(C);
    compute_eg_L(C);
    C->sX.alloc((size_t)n * d);
    C->sY.alloc((size_t)n * d);
    C->sXf.alloc((size_t)l * d);
    C->sYf.alloc((size_t)l * d);
    KOT_CUDA(cudaMemcpyAsync(C->sX.p, dX, (size_t)n * d * sizeof(double), cudaMemcpyDeviceToDevice, st));
    KOT_CUDA(cudaMemcpyAsync(C->sY.p, dY, (size_t)n * d * sizeof(double), cudaMemcpyDeviceToDevice, st));
    KOT_CUDA(cudaMemcpyAsync(C->sXf.p, dXf, (size_t)l * d * sizeof(double), cudaMemcpyDeviceToDevice, st));
    KOT_CUDA(cudaMemcpyAsync(C->sYf.p, dYf, (size_t)l * d * sizeof(double), cudaMemcpyDeviceToDevice, st));
    KOT_CUDA(cudaStreamSynchronize(st));
    C->d = d;
    C->n = n;
    C->sigma = sigma;
    C->have_samples = true;
    C->have = true;
  });
}

kot_status kot_set_features(kot_ctx* C, int l, const double* Q, const double* z, double q2,
                            const double* R, double lambda1, double lambda2) {
  if (!C) return KOT_ERR_INVALID;
  if (l < 1 || l > 32768 || !Q || !z || !R || !std::isfinite(q2) || !pos_finite(lambda1) ||
      !pos_finite(lambda2)) {
    C->err = "kot_set_features: invalid argument";
    return KOT_ERR_INVALID;
  }
  return run(C, [&] {
    KOT_CUDA(cudaSetDevice(C->opt.device));
    C->have = false;
    C->have_samples = false;
    C->l = l;
    ensure(C, l);
    reset_slots(C);
    const size_t L2 = (size_t)l * l;
    const double* dQ = dev_in(C, 0, Q, L2);
    const double* dz = dev_in(C, 1, z, l);
    const double* dR = dev_in(C, 2, R, L2);
    copy_mat(C->st, l, l, dQ, l, C->Q.p, l);
    KOT_CUDA(cudaMemcpyAsync(C->z.p, dz, l * sizeof(double), cudaMemcpyDeviceToDevice, C->st));
    KOT_CUDA(cudaMemcpyAsync(C->w_mu.p, dz, l * sizeof(double), cudaMemcpyDeviceToDevice, C->st));
    fill(C->st, l, 0.0, C->w_nu.p);
    fill(C->st, l, 0.0, C->c.p);
    copy_mat(C->st, l, l, dR, l, C->R.p, l);
    zero_lower(C->st, l, C->R.p);                        // rows below the diagonal ignored
    gemm_f64(C->st, true, false, l, l, l, 1.0, C->R.p, l, C->R.p, l, nullptr, 0.0, C->K.p, l,
             G_KHI_ROW | G_KHI_COL | G_SYM);             // K = R^T R
    C->q2 = q2;
    C->lambda1 = lambda1;
    C->lambda2 = lambda2;
    C->eps = 0.0;
    compute_eg_L(C);
    C->have = true;
  });
}

kot_status kot_get_features(kot_ctx* C, double* Q, double* K, double* R, double* z, double* w_mu,
                            double* w_nu, double* c, double* q2, double* eps) {
  if (!C) return KOT_ERR_INVALID;
  if (!C->have) {
    C->err = "kot_get_features: no features";
    return KOT_ERR_STATE;
  }
  return run(C, [&] {
    KOT_CUDA(cudaSetDevice(C->opt.device));
    const int l = C->l;
    const size_t L2 = (size_t)l * l;
    dev_out(C, Q, C->Q.p, L2);
    dev_out(C, K, C->K.p, L2);
    dev_out(C, R, C->R.p, L2);
    dev_out(C, z, C->z.p, l);
    dev_out(C, w_mu, C->w_mu.p, l);
    dev_out(C, w_nu, C->w_nu.p, l);
    dev_out(C, c, C->c.p, l);
    C->hs[0] = C->q2;
    C->hs[1] = C->eps;
    if (q2) KOT_CUDA(cudaMemcpyAsync(q2, C->hs, sizeof(double), cudaMemcpyDefault, C->st));
    if (eps) KOT_CUDA(cudaMemcpyAsync(eps, C->hs + 1, sizeof(double), cudaMemcpyDefault, C->st));
    KOT_CUDA(cudaStreamSynchronize(C->st));
  });
}

kot_status kot_residual(kot_ctx* C, const double* gamma, const double* X, double* r1, double* r2,
                        double* proj, double* sig, double* norms) {
  if (!C) return KOT_ERR_INVALID;
  if (!gamma || !X) {
    C->err = "kot_residual: gamma and X are required";
    return KOT_ERR_INVALID;
  }
  if (!C->have) {
    C->err = "kot_residual: no features";
    return KOT_ERR_STATE;
  }
  return run(C, [&] {
    KOT_CUDA(cudaSetDevice(C->opt.device));
    const int l = C->l;
    const size_t L2 = (size_t)l * l;
    const double* dg = dev_in(C, 0, gamma, l);
    const double* dXm = dev_in(C, 1, X, L2);
    residual(C, dg, dXm, C->ew, nullptr, C->rw);
    dev_out(C, r1, C->rw.r1.p, l);
    dev_out(C, r2, C->rw.r2.p, L2);
    dev_out(C, proj, C->M2.p, L2);
    dev_out(C, sig, C->ew.sig.p, l);
    if (norms) {
      double h[3] = {C->rw.n1, C->rw.n2, C->rw.norm};
      KOT_CUDA(cudaMemcpyAsync(norms, h, sizeof(h), cudaMemcpyDefault, C->st));
    }
    KOT_CUDA(cudaStreamSynchronize(C->st));
  });
}

kot_status kot_newton_direction(kot_ctx* C, const double* gamma, const double* X, double mu,
                                double cg_tol_abs, double* dgamma, double* dX, int* cg_iters) {
  if (!C) return KOT_ERR_INVALID;
  if (!gamma || !X || !dgamma || !dX || !pos_finite(mu) || !std::isfinite(cg_tol_abs)) {
    C->err = "kot_newton_direction: invalid argument";
    return KOT_ERR_INVALID;
  }
  if (!C->have) {
    C->err = "kot_newton_direction: no features";
    return KOT_ERR_STATE;
  }
  return run(C, [&] {
    KOT_CUDA(cudaSetDevice(C->opt.device));
    const int l = C->l;
    const size_t L2 = (size_t)l * l;
    const double* dg = dev_in(C, 0, gamma, l);
    const double* dXm = dev_in(C, 1, X, L2);
    residual(C, dg, dXm, C->ew, nullptr, C->rw);
    const int it = newton_direction(C, C->rw, C->ew, mu, cg_tol_abs, C->dg.p, C->dX.p, true);
    dev_out(C, dgamma, C->dg.p, l);
    dev_out(C, dX, C->dX.p, L2);
    KOT_CUDA(cudaStreamSynchronize(C->st));
    if (cg_iters) *cg_iters = it;
  });
}

kot_status kot_eig_sym(kot_ctx* C, int l, const double* Z, const double* warm, double* P,
                       double* sig, int* info) {
  if (!C) return KOT_ERR_INVALID;
  if (l < 1 || !Z || !P || !sig) {
    C->err = "kot_eig_sym: invalid argument";
    return KOT_ERR_INVALID;
  }
  return run(C, [&] {
    KOT_CUDA(cudaSetDevice(C->opt.device));
    const size_t L2 = (size_t)l * l;
    const double* dZ = dev_in(C, 0, Z, L2);
    const double* dW = warm ? dev_in(C, 1, warm, L2) : nullptr;
    C->eZ.alloc(L2);
    C->eP.alloc(L2);
    C->esig.alloc((size_t)l);
    copy_mat(C->st, l, l, dZ, l, C->eZ.p, l);
    symmetrize(C->st, l, C->eZ.p);
    C->jw.refine_done = 1e-8;   // the building block always refines to FP64 rounding
    eig_sym_f64(C->st, l, C->eZ.p, dW, C->eP.p, C->esig.p, C->jw, kMaxSweeps, C->hs,
                C->opt.eig_ctas, C->opt.eig_refine);
    dev_out(C, P, C->eP.p, L2);
    dev_out(C, sig, C->esig.p, l);
    KOT_CUDA(cudaStreamSynchronize(C->st));
    if (info) {
      info[0] = C->jw.last_sweeps;
      info[1] = C->jw.last_refine;
    }
  });
}

kot_status kot_ssn_solve(kot_ctx* C, double tol, double* gamma_out, double* X_out,
                         const double* gamma0, const double* X0, kot_result* res) {
  if (!C) return KOT_ERR_INVALID;
  if (!gamma_out || !pos_finite(tol)) {
    C->err = "kot_ssn_solve: invalid argument";
    return KOT_ERR_INVALID;
  }
  if (!C->have) {
    C->err = "kot_ssn_solve: no features";
    return KOT_ERR_STATE;
  }
  const auto t0 = std::chrono::steady_clock::now();
  kot_result R{};
  bool converged = false;
  kot_status s = run(C, [&] {
    KOT_CUDA(cudaSetDevice(C->opt.device));
    const int l = C->l;
    const size_t L2 = (size_t)l * l;
    cudaStream_t st = C->st;
    const kot_options& o = C->opt;
    reset_slots(C);
    C->in_solve = true;   // cross-sequence warm starts (eig_into) within this solve
    C->eig_calls = C->eig_sweeps = C->eig_refined = C->eig_refine_steps = 0;
    if (gamma0) {
      const double* p = dev_in(C, 0, gamma0, l);
      KOT_CUDA(cudaMemcpyAsync(C->g.p, p, l * sizeof(double), cudaMemcpyDeviceToDevice, st));
    } else {
      fill(st, l, 0.0, C->g.p);
    }
    if (X0) {
      const double* p = dev_in(C, 1, X0, L2);
      KOT_CUDA(cudaMemcpyAsync(C->X.p, p, L2 * sizeof(double), cudaMemcpyDeviceToDevice, st));
    } else {
      fill(st, L2, 0.0, C->X.p);
    }
    KOT_CUDA(cudaMemcpyAsync(C->vg.p, C->g.p, l * sizeof(double), cudaMemcpyDeviceToDevice, st));
    KOT_CUDA(cudaMemcpyAsync(C->vX.p, C->X.p, L2 * sizeof(double), cudaMemcpyDeviceToDevice, st));
    double theta = o.theta0;
    const double eta = o.eg_step > 0 ? o.eg_step : 1.0 / C->eg_L;
    residual(C, C->g.p, C->X.p, C->ew, nullptr, C->rw);
    C->hist.clear();
    C->trace.clear();
    if (o.record_history) C->hist.push_back(C->rw.norm);
    // the EG sequence v (its own context, stream and helper thread) from v0 = w0
    kot_ctx* V = o.use_eg ? lane_for_solve(C) : nullptr;
    int it = 0, acc = 0, egt = 0, cgt = 0;
    while (C->rw.norm > tol && it < o.max_iter) {
      LaneJoin join;
      if (V) {
        lane_start(C, eta);   // one EG step on v and R(v), beside the Newton step below
        join.C = C;
      }
      const double mu = theta * C->rw.norm;
      // mixed form: tensor-core products far from the solution, FP64 near it
      const int cgk = newton_direction(C, C->rw, C->ew, mu, 0.0, C->dg.p, C->dX.p,
                                       C->rw.norm > o.mixed_switch);
      cgt += cgk;
      axpby(st, l, 1.0, C->g.p, 1.0, C->dg.p, C->tg.p);
      axpby(st, L2, 1.0, C->X.p, 1.0, C->dX.p, C->tX.p);
      if (V && !C->plast_valid) {
        // no basis of its own yet (w0 = 0 gives a diagonal Z): wait for the EG projections and
        // start R(w~) from the lane's latest basis instead of cold Jacobi sweeps
        join.C = nullptr;
        lane_wait(C);
        if (V->plast_valid) {
          KOT_CUDA(cudaMemcpyAsync(C->Plast.p, V->Plast.p, L2 * sizeof(double), cudaMemcpyDeviceToDevice, st));
          C->plast_valid = true;
          KOT_CUDA(cudaEventRecord(C->lane_ev, st));
        }
      }
      residual(C, C->tg.p, C->tX.p, C->et, &C->ew, C->rt, false, true);
      pair_inner(C, C->rt, C->dg.p, C->dX.p);
      fetch(C, 6);
      finish_residual(C, C->rt);
      if (V && join.C) {
        join.C = nullptr;
        lane_wait(C);
      }
      const double inner = C->hs[2] + C->hs[3];
      const double dwn = std::sqrt(C->hs[4]) + std::sqrt(C->hs[5]);
      const double rho = -inner;
      if (rho >= o.alpha2 * dwn * dwn) theta = std::max(o.theta_min, o.beta0 * theta);
      else if (rho >= o.alpha1 * dwn * dwn) theta = o.beta1 * theta;
      else theta = std::min(o.theta_max, o.beta2 * theta);
      if (!V || C->rt.norm <= V->rv.norm) {
        std::swap(C->g, C->tg);
        std::swap(C->X, C->tX);
        swap_res(C->rw, C->rt);
        swap_slots(C->ew, C->et);
        ++acc;
      } else {
        // w = v: the iterate, its residual and its eigen-decomposition copied out of the lane
        // (whose stream is idle after R(v)); the lane's next step waits for these reads
        KOT_CUDA(cudaMemcpyAsync(C->g.p, V->vg.p, l * sizeof(double), cudaMemcpyDeviceToDevice, st));
        KOT_CUDA(cudaMemcpyAsync(C->X.p, V->vX.p, L2 * sizeof(double), cudaMemcpyDeviceToDevice, st));
        KOT_CUDA(cudaMemcpyAsync(C->rw.r1.p, V->rv.r1.p, l * sizeof(double), cudaMemcpyDeviceToDevice, st));
        KOT_CUDA(cudaMemcpyAsync(C->rw.r2.p, V->rv.r2.p, L2 * sizeof(double), cudaMemcpyDeviceToDevice, st));
        C->rw.n1 = V->rv.n1;
        C->rw.n2 = V->rv.n2;
        C->rw.norm = V->rv.norm;
        KOT_CUDA(cudaMemcpyAsync(C->ew.P.p, V->ev.P.p, L2 * sizeof(double), cudaMemcpyDeviceToDevice, st));
        KOT_CUDA(cudaMemcpyAsync(C->ew.sig.p, V->ev.sig.p, l * sizeof(double), cudaMemcpyDeviceToDevice, st));
        C->ew.nb = V->ev.nb;
        C->ew.valid = V->ev.valid;
        C->ew.trivial = V->ev.trivial;
        KOT_CUDA(cudaEventRecord(C->lane_ev, st));
        ++egt;
      }
      ++it;
      if (o.record_history) {
        C->hist.push_back(C->rw.norm);
        for (double v : {C->rw.norm, mu, (double)cgk, theta, (double)C->last_dir_kind}) C->trace.push_back(v);
      }
    }
    converged = C->rw.norm <= tol;
    double ot = 0;
    const double obj = objective_and_ot(C, C->g.p, &ot);
    dev_out(C, gamma_out, C->g.p, l);
    dev_out(C, X_out, C->X.p, L2);
    KOT_CUDA(cudaStreamSynchronize(st));
    R.iters = it;
    R.ssn_accepted = acc;
    R.eg_taken = egt;
    R.cg_total = cgt;
    R.residual = C->rw.norm;
    R.r1_norm = C->rw.n1;
    R.r2_norm = C->rw.n2;
    R.objective = obj;
    R.ot_hat = ot;
    R.eps = C->eps;
    R.eig_calls = (int)C->eig_calls;
    R.eig_sweeps = (int)C->eig_sweeps;
    R.eig_refined = (int)C->eig_refined;
    R.eig_refine_steps = (int)C->eig_refine_steps;
    if (V) {
      R.eig_calls += (int)V->eig_calls;
      R.eig_sweeps += (int)V->eig_sweeps;
      R.eig_refined += (int)V->eig_refined;
      R.eig_refine_steps += (int)V->eig_refine_steps;
    }
  });
  if (s == KOT_OK && !converged) {
    s = KOT_ERR_NO_CONVERGENCE;
    C->err = "kot_ssn_solve: iteration cap reached";
  }
  R.status = s;
  R.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (res) *res = R;
  return s;
}

kot_status kot_eg_solve(kot_ctx* C, double tol, double* gamma_out, double* X_out, const double* gamma0,
                        const double* X0, kot_result* res) {
  if (!C) return KOT_ERR_INVALID;
  if (!gamma_out || !pos_finite(tol)) {
    C->err = "kot_eg_solve: invalid argument";
    return KOT_ERR_INVALID;
  }
  if (!C->have) {
    C->err = "kot_eg_solve: no features";
    return KOT_ERR_STATE;
  }
  const auto t0 = std::chrono::steady_clock::now();
  kot_result R{};
  bool converged = false;
  kot_status s = run(C, [&] {
    KOT_CUDA(cudaSetDevice(C->opt.device));
    const int l = C->l;
    const size_t L2 = (size_t)l * l;
    cudaStream_t st = C->st;
    const kot_options& o = C->opt;
    reset_slots(C);
    C->in_solve = true;   // cross-sequence warm starts (eig_into) within this solve
    C->eig_calls = C->eig_sweeps = C->eig_refined = C->eig_refine_steps = 0;
    if (gamma0) {
      const double* p = dev_in(C, 0, gamma0, l);
      KOT_CUDA(cudaMemcpyAsync(C->vg.p, p, l * sizeof(double), cudaMemcpyDeviceToDevice, st));
    } else {
      fill(st, l, 0.0, C->vg.p);
    }
    if (X0) {
      const double* p = dev_in(C, 1, X0, L2);
      KOT_CUDA(cudaMemcpyAsync(C->vX.p, p, L2 * sizeof(double), cudaMemcpyDeviceToDevice, st));
    } else {
      fill(st, L2, 0.0, C->vX.p);
    }
    const double eta = o.eg_step > 0 ? o.eg_step : 1.0 / C->eg_L;
    residual(C, C->vg.p, C->vX.p, C->ev, nullptr, C->rv, true);
    C->hist.clear();
    C->trace.clear();
    if (o.record_history) C->hist.push_back(C->rv.norm);
    int it = 0;
    while (C->rv.norm > tol && it < o.max_iter) {
      eg_step(C, eta);
      residual(C, C->vg.p, C->vX.p, C->ev, &C->ev, C->rv, true);
      ++it;
      if (o.record_history) C->hist.push_back(C->rv.norm);
    }
    converged = C->rv.norm <= tol;
    double ot = 0;
    const double obj = objective_and_ot(C, C->vg.p, &ot);
    dev_out(C, gamma_out, C->vg.p, l);
    dev_out(C, X_out, C->vX.p, L2);
    KOT_CUDA(cudaStreamSynchronize(st));
    R.iters = it;
    R.eg_taken = it;
    R.residual = C->rv.norm;
    R.r1_norm = C->rv.n1;
    R.r2_norm = C->rv.n2;
    R.objective = obj;
    R.ot_hat = ot;
    R.eps = C->eps;
    R.eig_calls = (int)C->eig_calls;
    R.eig_sweeps = (int)C->eig_sweeps;
    R.eig_refined = (int)C->eig_refined;
    R.eig_refine_steps = (int)C->eig_refine_steps;
  });
  if (s == KOT_OK && !converged) {
    s = KOT_ERR_NO_CONVERGENCE;
    C->err = "kot_eg_solve: iteration cap reached";
  }
  R.status = s;
  R.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (res) *res = R;
  return s;
}

kot_status kot_potentials(kot_ctx* C, int side, int m, const double* points, const double* gamma,
                          double* u, double* grad, double* tmap) {
  if (!C) return KOT_ERR_INVALID;
  if ((side != 0 && side != 1) || m < 1 || !points || !gamma || (!u && !grad && !tmap)) {
    C->err = "kot_potentials: invalid argument";
    return KOT_ERR_INVALID;
  }
  if (!C->have || !C->have_samples) {
    C->err = "kot_potentials: needs the samples of kot_build_features";
    return KOT_ERR_STATE;
  }
  return run(C, [&] {
    KOT_CUDA(cudaSetDevice(C->opt.device));
    const int d = C->d, l = C->l;
    const double* dP = dev_in(C, 0, points, (size_t)m * d);
    const double* dg = dev_in(C, 1, gamma, (size_t)l);
    double *du = u, *dgr = grad, *dt = tmap;
    if (C->opt.host_pointers) {
      C->stage[2].alloc((size_t)m);
      C->stage[3].alloc((size_t)m * d);
      C->stage[4].alloc((size_t)m * d);
      du = u ? C->stage[2].p : nullptr;
      dgr = grad ? C->stage[3].p : nullptr;
      dt = tmap ? C->stage[4].p : nullptr;
    }
    potential_f64(C->st, m, d, C->n, side == 0 ? C->sX.p : C->sY.p, l, side == 0 ? C->sXf.p : C->sYf.p, dg,
                  dP, C->sigma, C->lambda2, du, dgr, dt);
    if (C->opt.host_pointers) {
      dev_out(C, u, du, (size_t)m);
      dev_out(C, grad, dgr, (size_t)m * d);
      dev_out(C, tmap, dt, (size_t)m * d);
    }
    KOT_CUDA(cudaStreamSynchronize(C->st));
  });
}

namespace {
// Pseudo-random entries in [-1, 1) from an integer hash of the index (inputs for the autotuner)
__global__ void k_fill_hash(size_t n, unsigned seed, double* __restrict__ out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    unsigned x = (unsigned)i * 2654435761u ^ seed;
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    out[i] = (double)x * (2.0 / 4294967296.0) - 1.0;
  }
}
}  // namespace

kot_status kot_autotune(kot_ctx* C, int l, int* choice) {
  if (!C) return KOT_ERR_INVALID;
  if (l < 1 || l > 32768) {
    C->err = "kot_autotune: invalid argument";
    return KOT_ERR_INVALID;
  }
  return run(C, [&] {
    KOT_CUDA(cudaSetDevice(C->opt.device));
    cudaStream_t st = C->st;
    const int dev = C->opt.device;
    const size_t L2 = (size_t)l * l;
    DevBuf<double> A, B, Cm, P, sig;
    A.alloc(L2);
    B.alloc(L2);
    Cm.alloc(L2);
    P.alloc(L2);
    sig.alloc((size_t)l);
    const int fb = (int)std::min<size_t>((L2 + 255) / 256, 1216);
    k_fill_hash<<<fb, 256, 0, st>>>(L2, 12345u, A.p);
    k_fill_hash<<<fb, 256, 0, st>>>(L2, 67890u, B.p);
    KOT_LAUNCHED(2);
    KOT_CUDA(cudaPeekAtLastError());
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    KOT_CUDA(cudaEventCreate(&e0));
    KOT_CUDA(cudaEventCreate(&e1));
    struct EventGuard {
      cudaEvent_t a, b;
      ~EventGuard() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
      }
    } guard{e0, e1};
    auto timed = [&](const std::function<void()>& f, int reps) -> float {
      f();                                   // warm (buffers, descriptors, caches)
      KOT_CUDA(cudaEventRecord(e0, st));
      for (int r = 0; r < reps; ++r) f();
      KOT_CUDA(cudaEventRecord(e1, st));
      KOT_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      KOT_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      return ms / reps;
    };
    int best_split[2] = {0, 0}, best_bn[2] = {64, 64};
    const int slices[2] = {3, 6};
    for (int q = 0; q < 2; ++q) {
      float best = 1e30f;
      for (int bn : {64, 128})
        for (int S : {1, 2, 3, 4, 6, 8, 12, 16}) {
          C->oz.splits_override = S;
          C->oz.bn_override = bn;
          const float t = timed([&] {
            gemm_oz(st, C->oz, l, l, l, TcOperand{A.p, l, false, nullptr}, TcOperand{B.p, l, true, nullptr},
                    slices[q], 1.0, 0.0, Cm.p, l, false);
          }, 5);
          if (t < best) {
            best = t;
            best_split[q] = S;
            best_bn[q] = bn;
          }
        }
      C->oz.splits_override = 0;
      C->oz.bn_override = 0;
      set_tuned_splits(dev, l, slices[q], best_split[q]);
      set_tuned_tile_width(dev, l, slices[q], best_bn[q]);
    }
    if (gemm_oz_error(st, C->oz)) fail(KOT_ERR_TIMEOUT, "tensor-core FP64-emulation wait timed out");
    // cooperative Jacobi: CTA count for a cold decomposition of a symmetric l x l matrix
    axpby(st, L2, 1.0, A.p, 0.0, nullptr, Cm.p);
    symmetrize(st, l, Cm.p);
    int nsm = 152;
    KOT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    int best_ctas = nsm, best_threads = 512;
    float best = 1e30f;
    std::vector<double> sig0, sig1((size_t)l);
    for (int threads : {256, 512, 1024})
      for (int ctas : {nsm / 4, nsm / 2, nsm}) {
        if (ctas < 1) continue;
        C->jw.threads_override = threads;
        const float t = timed([&] {
          eig_sym_f64(st, l, Cm.p, nullptr, P.p, sig.p, C->jw, kMaxSweeps, C->hs, ctas, 0);
        }, 1);
        // a launch shape is a candidate only if it gives the first shape's eigenvalues
        KOT_CUDA(cudaMemcpyAsync(sig1.data(), sig.p, (size_t)l * sizeof(double), cudaMemcpyDeviceToHost, st));
        KOT_CUDA(cudaStreamSynchronize(st));
        if (sig0.empty()) sig0 = sig1;
        double scale = 0.0, diff = 0.0;
        for (int i = 0; i < l; ++i) {
          scale = std::max(scale, std::fabs(sig0[i]));
          diff = std::max(diff, std::fabs(sig1[i] - sig0[i]));
        }
        if (!(diff <= 1e-12 * std::max(scale, 1e-300))) continue;
        if (t < best) {
          best = t;
          best_ctas = ctas;
          best_threads = threads;
        }
      }
    C->jw.threads_override = 0;
    set_tuned_jacobi_ctas(dev, l, best_ctas);
    set_tuned_jacobi_threads(dev, l, best_threads);
    if (choice) {
      choice[0] = best_split[0];
      choice[1] = best_split[1];
      choice[2] = best_ctas;
      choice[3] = best_bn[0];
      choice[4] = best_bn[1];
      choice[5] = best_threads;
    }
    for (DevBuf<double>* b : {&A, &B, &Cm, &P, &sig}) b->release();
  });
}

kot_status kot_dense_product(kot_ctx* C, int M, int N, int K, double alpha, const double* A,
                             int lda, int transA, const double* B, int ldb, int transB,
                             double beta, double* Cm, int ldc, int pieces) {
  if (!C) return KOT_ERR_INVALID;
  if (M < 1 || N < 1 || K < 1 || !A || !B || !Cm || pieces < -8 || pieces > 3 || pieces == -1 ||
      pieces == -2 ||
      lda < (transA ? M : K) || ldb < (transB ? N : K) || ldc < N || !std::isfinite(alpha) ||
      !std::isfinite(beta)) {
    C->err = "kot_dense_product: invalid argument";
    return KOT_ERR_INVALID;
  }
  return run(C, [&] {
    KOT_CUDA(cudaSetDevice(C->opt.device));
    const size_t na = (size_t)(transA ? K : M) * lda, nb = (size_t)(transB ? K : N) * ldb;
    const double* dA = dev_in(C, 0, A, na);
    const double* dB = dev_in(C, 1, B, nb);
    double* dC = Cm;
    if (C->opt.host_pointers) {
      C->stage[2].alloc((size_t)M * ldc);
      KOT_CUDA(cudaMemcpyAsync(C->stage[2].p, Cm, (size_t)M * ldc * sizeof(double), cudaMemcpyHostToDevice, C->st));
      dC = C->stage[2].p;
    }
    if (pieces == 0) {
      // FP64 pipes: gemm_f64 takes op(B) as K x N, i.e. the transpose of this call's op(B)
      gemm_f64(C->st, transA != 0, transB == 0, M, N, K, alpha, dA, lda, dB, ldb, nullptr, beta, dC,
               ldc, 0);
    } else if (pieces < 0) {
      gemm_oz(C->st, C->oz, M, N, K, TcOperand{dA, lda, transA != 0, nullptr},
              TcOperand{dB, ldb, transB != 0, nullptr}, -pieces, alpha, beta, dC, ldc, false);
    } else {
      gemm_tc(C->st, C->tc, M, N, K, TcOperand{dA, lda, transA != 0, nullptr},
              TcOperand{dB, ldb, transB != 0, nullptr}, pieces, alpha, beta, dC, ldc);
    }
    if (C->opt.host_pointers) dev_out(C, Cm, dC, (size_t)M * ldc);
    KOT_CUDA(cudaStreamSynchronize(C->st));
    if (pieces > 0 && gemm_tc_error(C->st, C->tc)) fail(KOT_ERR_TIMEOUT, "tensor-core GEMM wait timed out");
    if (pieces < 0 && gemm_oz_error(C->st, C->oz)) fail(KOT_ERR_TIMEOUT, "tensor-core GEMM wait timed out");
  });
}

kot_status kot_wait_probe(kot_ctx* C, long long polls) {
  if (!C) return KOT_ERR_INVALID;
  if (polls < 1 || polls > 100000000LL) {
    C->err = "kot_wait_probe: polls must be in 1..1e8";
    return KOT_ERR_INVALID;
  }
  kot_status s = run(C, [&] {
    KOT_CUDA(cudaSetDevice(C->opt.device));
    if (starved_wait_probe(C->st, C->tc, polls)) fail(KOT_ERR_TIMEOUT, "bounded device wait gave up (probe)");
  });
  return s;
}

kot_status kot_launch_count(long long* out) {
  if (!out) return KOT_ERR_INVALID;
  *out = launch_total();
  return KOT_OK;
}

kot_status kot_profile(kot_ctx* C, int mask) {
  if (!C || mask < 0) return KOT_ERR_INVALID;
  return run(C, [&] {
    KOT_CUDA(cudaSetDevice(C->opt.device));
    C->prof.reset();
    C->prof.mask = mask;
  });
}

kot_status kot_profile_every(kot_ctx* C, int every) {
  if (!C || every < 1) return KOT_ERR_INVALID;
  return run(C, [&] {
    C->prof.reset();
    C->prof.every = every;
  });
}

kot_status kot_profile_read(kot_ctx* C, int cls, kot_kernel_stats* out) {
  if (!C || !out || cls < 0 || cls >= KC_COUNT) return KOT_ERR_INVALID;
  return run(C, [&] {
    C->prof.collect();
    out->launches = C->prof.launches[cls];
    out->ms = C->prof.ms[cls];
    out->flops = C->prof.flops[cls];
    out->bytes = C->prof.bytes[cls];
    out->exec_flops = C->prof.exec[cls];
  });
}

kot_status kot_get_trace(kot_ctx* C, double* out, int cap, int* count) {
  if (!C || !out || cap < 0 || !count) return KOT_ERR_INVALID;
  const int rows = std::min<int>(cap, (int)(C->trace.size() / 5));
  std::copy(C->trace.begin(), C->trace.begin() + 5 * rows, out);
  *count = rows;
  return KOT_OK;
}

kot_status kot_get_history(kot_ctx* C, double* hist, int cap, int* count) {
  if (!C || !hist || cap < 0 || !count) return KOT_ERR_INVALID;
  const int m = std::min<int>(cap, (int)C->hist.size());
  std::copy(C->hist.begin(), C->hist.begin() + m, hist);
  *count = m;
  return KOT_OK;
}

kot_status kot_bootstrap_solve(kot_ctx* C, int B, int n, const double* Xs, const double* Ys, double tol,
                               double* gamma_out, kot_result* res) {
  if (!C) return KOT_ERR_INVALID;
  if (B < 0 || n < 1 || (B > 0 && (!Xs || !Ys || !gamma_out || !res)) || !pos_finite(tol)) {
    C->err = "kot_bootstrap_solve: invalid argument";
    return KOT_ERR_INVALID;
  }
  if (!C->have || !C->have_samples) {
    C->err = "kot_bootstrap_solve: needs the filling points of kot_build_features";
    return KOT_ERR_STATE;
  }
  kot_status first = KOT_OK;
  const int d = C->d, l = C->l;
  for (int b = 0; b < B; ++b) {
    // the resample's sample terms of the dual problem (Sec. 3): w_mu, w_nu, q2 and z; Q, K, R,
    // the jitter and the EG step bound depend on the filling points only and are kept
    kot_status s = run(C, [&] {
      KOT_CUDA(cudaSetDevice(C->opt.device));
      cudaStream_t st = C->st;
      const size_t nd = (size_t)n * d;
      const double* dX = dev_in(C, 0, Xs + (size_t)b * nd, nd);
      const double* dY = dev_in(C, 1, Ys + (size_t)b * nd, nd);
      const double inv2s2 = 1.0 / (2.0 * C->sigma * C->sigma);
      embed_f64(st, n, d, l, dX, C->sXf.p, inv2s2, C->w_mu.p);
      embed_f64(st, n, d, l, dY, C->sYf.p, inv2s2, C->w_nu.p);
      const int pb = pair_blocks(n);
      C->stage[7].alloc(pb);
      pair_mean_f64(st, n, d, dX, inv2s2, C->scal.p + 10, C->stage[7].p, pb);
      pair_mean_f64(st, n, d, dY, inv2s2, C->scal.p + 11, C->stage[7].p, pb);
      cost_z_f64(st, l, d, C->sXf.p, C->sYf.p, C->lambda2, C->w_mu.p, C->w_nu.p, C->c.p, C->z.p);
      // the samples the potentials use are the resample's
      C->sX.alloc(nd);
      C->sY.alloc(nd);
      KOT_CUDA(cudaMemcpyAsync(C->sX.p, dX, nd * sizeof(double), cudaMemcpyDeviceToDevice, st));
      KOT_CUDA(cudaMemcpyAsync(C->sY.p, dY, nd * sizeof(double), cudaMemcpyDeviceToDevice, st));
      KOT_CUDA(cudaMemcpyAsync(C->hs + 10, C->scal.p + 10, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
      KOT_CUDA(cudaStreamSynchronize(st));
      C->q2 = C->hs[10] + C->hs[11];
      C->n = n;
    });
    if (s != KOT_OK) {   // the resample's features failed: report it for this and the rest
      for (int r = b; r < B; ++r) {
        res[r] = kot_result{};
        res[r].status = s;
      }
      return first == KOT_OK ? s : first;
    }
    s = kot_ssn_solve(C, tol, gamma_out + (size_t)b * l, nullptr, nullptr, nullptr, &res[b]);
    if (first == KOT_OK && s != KOT_OK) first = s;
  }
  return first;
}

kot_status kot_batch_solve(kot_ctx* C, int B, const kot_problem* probs, kot_result* res) {
  if (!C) return KOT_ERR_INVALID;
  if (B < 0 || (B > 0 && (!probs || !res))) {
    C->err = "kot_batch_solve: invalid argument";
    return KOT_ERR_INVALID;
  }
  for (int i = 0; i < B; ++i) {
    const kot_problem& p = probs[i];
    if (p.d < 1 || p.n < 1 || p.l < 1 || !p.X || !p.Y || !p.Xf || !p.Yf || !p.gamma_out ||
        !pos_finite(p.sigma) || !pos_finite(p.lambda1) || !pos_finite(p.lambda2) ||
        !pos_finite(p.tol)) {
      C->err = "kot_batch_solve: invalid problem " + std::to_string(i);
      return KOT_ERR_INVALID;
    }
  }
  if (B == 0) return KOT_OK;
  // largest problems first (cost grows like l^3), handed out through a shared counter
  std::vector<int> order(B);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return probs[a].l > probs[b].l; });
  // Each problem is latency-bound on its own, so several run at once: W worker contexts, each
  // with its own stream and buffers, driven by one host thread each; their cooperative
  // eigensolver launches take a share of the SMs so that all of them fit at the same time.
  int W = C->opt.batch_workers > 0 ? C->opt.batch_workers : 4;
  W = std::max(1, std::min(W, B));
  int nsm = 152;
  cudaSetDevice(C->opt.device);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, C->opt.device);
  std::vector<kot_ctx*> workers(W, nullptr);
  for (int w = 0; w < W; ++w) {
    kot_options o = C->opt;
    o.stream = nullptr;
    o.batch_workers = 1;
    if (o.eig_ctas == 0) o.eig_ctas = std::max(8, nsm / W);
    kot_status s = kot_create(&workers[w], &o);
    if (s != KOT_OK) {
      for (kot_ctx* x : workers) kot_destroy(x);
      C->err = "kot_batch_solve: could not create worker contexts";
      return s;
    }
  }
  std::atomic<int> next{0};
  auto work = [&](kot_ctx* X) {
    for (int k = next.fetch_add(1); k < B; k = next.fetch_add(1)) {
      const int i = order[k];
      const kot_problem& p = probs[i];
      kot_status s = kot_build_features(X, p.d, p.n, p.X, p.Y, p.l, p.Xf, p.Yf, p.sigma, p.lambda1,
                                        p.lambda2);
      if (s == KOT_OK) s = kot_ssn_solve(X, p.tol, p.gamma_out, nullptr, nullptr, nullptr, &res[i]);
      else {
        res[i] = kot_result{};
        res[i].status = s;
      }
    }
  };
  std::vector<std::thread> threads;
  for (int w = 1; w < W; ++w) threads.emplace_back(work, workers[w]);
  work(workers[0]);
  for (auto& t : threads) t.join();
  for (kot_ctx* x : workers) kot_destroy(x);
  kot_status first = KOT_OK;
  for (int i = 0; i < B && first == KOT_OK; ++i)
    if (res[i].status != KOT_OK) first = (kot_status)res[i].status;
  return first;
}

}  // extern "C"
