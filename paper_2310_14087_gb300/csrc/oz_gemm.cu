// FP64-accurate dense products on the tcgen05 tensor cores:
//   C = alpha * opA(A) * opB(B)^T + beta * C,   FP64 in, FP64 out,
// computed from exact BF16 x BF16 products summed exactly in FP32 (the splitting idea of Ozaki,
// Ogita and Oishi, Numer. Algorithms 59, 2012: cut each operand into fixed-point slices whose
// pairwise products are error-free on a low-precision multiplier, multiply slice by slice, and
// add the partial products in higher precision).
//
// Why: this GPU issues about two FP64 FMAs per clock per SM (1.2 TFLOP/s in all), so every
// O(l^3) FP64 product of the mixed form would otherwise run at ~1/1600 of the BF16 tensor rate.
//
// Slicing.  Logical row r of an operand (its K values, times the optional scale vector) has
// binary exponent e_r with max_k |v(r,k)| < 2^e_r.  Each value is rounded to the fixed-point
// integer X = round(|v| 2^(7 + 8 (s - 1) - e_r)) and X is written in balanced base-256 digits
// d_0 .. d_(s-1) with |d_i| <= 128, so that
//     v ~ 2^(e_r - 7) * sum_i d_i 2^(-8 i)          (error <= 2^(e_r - 8 s) per value).
// Slice i holds the BF16 value d_i 2^(-8 i), which is exact (at most 8 significant bits).
// The product of slice i of A and slice j of B ("level" t = i + j) is an integer of magnitude
// <= 2^14 times 2^(-8 t).  Levels t >= s are dropped (they are below the slicing error).
//
// Exact accumulation.  Terms of one level summed in FP32 stay exact while the integer sum stays
// <= 2^24, i.e. for up to 1024 products; the kernel closes an accumulation group after at most
// OZ_EXACT_TILES x 64 = 512 of them and never mixes levels in a group for t < OZ_EXACT_LEVELS.
// Levels >= OZ_EXACT_LEVELS (weight <= 2^-32 of level 0) share one FP32 group: its rounding is
// far below the slicing error.  Each finished group is read out of tensor memory and added to a
// float-float (hi, lo) pair per output element with an error-free two-sum, so the combination of
// groups costs FP32 additions only (FP64 would cost a clock per two elements on this part).
// Net accuracy: about 2^-47 relative to max_k |A(r,k)| * max_k |B(c,k)| * K per element for
// s = 6, i.e. FP64 GEMM accuracy up to a small factor.
//
// Kernels:
// (1) slicing into a BF16 operand matrix [rows][s * Kp] (slice i occupies columns i * Kp ..
//     i * Kp + Kp - 1). For K <= 2048 one launch: a thread-block cluster of <= 8 CTAs spans the K
//     range of 32 rows and exchanges per-row exponents through distributed shared memory. For
//     larger K, an exponent-partials kernel and a slicing kernel.
// (2) the tcgen05 GEMM, one CTA per output tile (128 x 64, or 128 x 128 when M, N >= 512) and
//     split z of the (slice pair, k tile) sequence:
//     * the TMA producer warp streams 128 x 64 (A) and BN x 64 (B) BF16 tiles into a 6-stage
//       ring;
//     * the MMA warp issues tcgen05.mma (M 128, N BN, K 16) into one of two BN-column FP32
//       accumulators in tensor memory and hands each finished group to the BN / 16 epilogue
//       warps (64 columns each), which drain it while the next group accumulates in the other
//       buffer;
//     * the (hi, lo) pairs of each split go, staged through the free operand ring, to a float2
//       buffer.
// (3) finalize: sum the splits, convert to FP64, scale by alpha 2^(e_r - 7) 2^(e_c - 7), add
//     beta C.  A symmetric result is stored from the entries on or above the diagonal, each at
//     both positions, so it is exactly symmetric; GEMM tiles wholly below the diagonal do nothing.
//     (Storing C from the GEMM epilogue instead, with one split, or adding the splits in the
//     last-arriving CTA, was measured slower: 34 vs 14 us at 300^3, 592 + 107 vs 519 + 186 us at
//     2048^3.)
// Every wait is bounded.
#include <cuda.h>
#include <cuda_bf16.h>

#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "kot_internal.cuh"
#include "oz_slicing.cuh"
#include "tc_ptx.cuh"

namespace kot {

namespace cg = cooperative_groups;

namespace {

constexpr int OZ_BM = 128, OZ_BK = 64, OZ_STAGES = 6;
constexpr int OZ_A_BYTES = OZ_BM * OZ_BK * 2;   // 16 KB

// Tile configuration by output-tile width BN (64 or 128): BN / 16 epilogue warps, each owning 64
// accumulator columns of one 32-lane quarter of tensor memory, then the TMA producer warp and
// the MMA warp.
template <int BN>
struct OzCfg {
  static constexpr int EPI = BN / 16;                       // epilogue warps
  static constexpr int THREADS = 32 * (EPI + 2);
  static constexpr int B_BYTES = BN * OZ_BK * 2;            // 8 or 16 KB
  static constexpr int STAGE = OZ_A_BYTES + B_BYTES;
  static constexpr int SMEM = OZ_STAGES * STAGE + 1024 + 256;
  static constexpr int TMEM_COLS = 2 * BN;                  // two accumulator buffers
  static_assert(EPI * 32 * 65 * 8 <= OZ_STAGES * STAGE, "epilogue staging fits in the ring");
};
constexpr int OZ_EXACT_LEVELS = oz::kExactLevels;
constexpr int OZ_EXACT_TILES = oz::kExactTiles;
constexpr int OZ_MAX_SLICES = oz::kMaxSlices;
constexpr int OZ_MAX_PAIRS = OZ_MAX_SLICES * (OZ_MAX_SLICES + 1) / 2;
constexpr int OZ_MAX_SPLITS = 16;
constexpr int kOzDefaultSplits = 8;
constexpr int kSplitRows = 16;        // thread rows of a cluster slicing block (32 x 16 threads)
constexpr int kOzClusterK = 8 * 256;  // K up to which one (portable, <= 8 CTA) cluster spans a row

inline int cdiv(size_t a, int b) { return (int)((a + b - 1) / b); }

static_assert(sizeof(CUtensorMap) == 128, "tensor map size");

// ordinal of the current device (0..63)
int device_index() {
  int dev = 0;
  KOT_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) throw Error{KOT_ERR_CUDA, "device ordinal out of range"};
  return dev;
}

// SM count of the current device, queried once per device
int sm_count() {
  static int cache[64] = {};
  const int dev = device_index();
  if (cache[dev] == 0) {
    int n = 0;
    KOT_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
    cache[dev] = n;
  }
  return cache[dev];
}

// Split counts and tile widths chosen by the autotuner, per device, size bucket (ceil log2 of
// max(M, N)) and slice count; 0 = not tuned.
int g_tuned_splits[64][32][OZ_MAX_SLICES + 1] = {};
int g_tuned_bn[64][32][OZ_MAX_SLICES + 1] = {};

int size_bucket(int mn) {
  int b = 0;
  while ((1 << b) < mn && b < 31) ++b;
  return b;
}

struct OzPlan {
  int M, N, Kp, nk, npairs, sym;
  int sbeg[OZ_MAX_SPLITS + 1];        // split z takes tile steps [sbeg[z], sbeg[z + 1])
  signed char pa[OZ_MAX_PAIRS], pb[OZ_MAX_PAIRS], lv[OZ_MAX_PAIRS];
  float2* W;                          // splits x M x N partial sums (hi, lo)
  int* err;
};

__device__ __forceinline__ bool oz_new_group(int prev, int lv, int gt) { return oz::new_group(prev, lv, gt); }

// (hi, lo) += g with Knuth's error-free two-sum on hi; rounding is pinned (no contraction).
__device__ __forceinline__ void ff_add(float& hi, float& lo, float g) {
  const float s = __fadd_rn(hi, g);
  const float bp = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(g, bp));
  hi = s;
  lo = __fadd_rn(lo, e);
}

template <int BN>
__global__ void __launch_bounds__(OzCfg<BN>::THREADS, 1)
    k_oz_gemm(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
              const __grid_constant__ OzPlan P) {
  using Cfg = OzCfg<BN>;
  constexpr int EPI = Cfg::EPI, OZ_STAGE = Cfg::STAGE, OZ_BN = BN;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + OZ_STAGES * OZ_STAGE);
  uint64_t* empty = full + OZ_STAGES;
  uint64_t* acc_full = empty + OZ_STAGES;   // [2]: group in buffer b is complete
  uint64_t* acc_empty = acc_full + 2;       // [2]: buffer b has been read out (4 warp arrivals)
  uint64_t* done = acc_empty + 2;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * OZ_BM, n0 = blockIdx.x * OZ_BN, z = blockIdx.z;
  if (P.sym && n0 + OZ_BN <= m0) {   // wholly below the diagonal: k_oz_finalize mirrors it
    pdl_wait();
    pdl_trigger();
    return;
  }
  const int nk = P.nk;
  // split z takes the tile steps [s0, s1) of the sequence (pair p, k tile kt), step = p nk + kt
  const int s0 = P.sbeg[z], s1 = P.sbeg[z + 1];

  if (threadIdx.x == 0) {
    for (int s = 0; s < OZ_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], EPI);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(tmem_slot, Cfg::TMEM_COLS);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  bool ok = true;
  // barrier set-up and the tensor-memory allocation above overlap the slicing kernel's tail
  pdl_wait();
  pdl_trigger();

  if (warp == EPI) {
    if (lane == 0) {
      // TMA producer: the tiles of this split's steps, in order (counters kept incrementally:
      // this thread is on the critical path)
      int p = s0 / nk, kt = s0 - p * nk, s = 0;
      uint32_t ph = 0;
      for (int n = s0; n < s1; ++n) {
        if (!mbar_wait(&empty[s], ph ^ 1u)) {
          ok = false;
          break;
        }
        mbar_expect_tx(&full[s], OZ_STAGE);
        uint8_t* st = smem + s * OZ_STAGE;
        tma_load_2d(st, &ta, &full[s], P.pa[p] * P.Kp + kt * OZ_BK, m0);
        tma_load_2d(st + OZ_A_BYTES, &tb, &full[s], P.pb[p] * P.Kp + kt * OZ_BK, n0);
        if (++kt == nk) {
          kt = 0;
          ++p;
        }
        if (++s == OZ_STAGES) {
          s = 0;
          ph ^= 1u;
        }
      }
    }
  } else if (warp == EPI + 1) {
    if (lane == 0) {
      // MMA issuer
      constexpr uint32_t idesc = idesc_bf16(OZ_BM, OZ_BN);
      int g = -1, gt = 0, prev = -1;
      int p = s0 / nk, kt = s0 - p * nk, s = 0;
      uint32_t ph = 0;
      for (int n = s0; n < s1; ++n) {
        const int lv = P.lv[p];
        const bool first = oz_new_group(prev, lv, gt);
        if (first) {
          if (g >= 0) umma_commit(&acc_full[g & 1]);
          ++g;
          gt = 0;
          // the buffer must have been read out (group g - 2) before it is overwritten
          if (!mbar_wait(&acc_empty[g & 1], (((uint32_t)g >> 1) & 1u) ^ 1u)) {
            ok = false;
            break;
          }
        }
        if (!mbar_wait(&full[s], ph)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a_addr = smem_u32(smem + s * OZ_STAGE);
        const uint32_t b_addr = a_addr + OZ_A_BYTES;
        const uint32_t d = tmem + (uint32_t)((g & 1) * OZ_BN);
#pragma unroll
        for (int k = 0; k < OZ_BK / 16; ++k)
          umma_bf16(d, smem_desc_sw128(a_addr + 32 * k), smem_desc_sw128(b_addr + 32 * k), idesc,
                    (first && k == 0) ? 0u : 1u);
        umma_commit(&empty[s]);
        ++gt;
        prev = lv;
        if (++kt == nk) {
          kt = 0;
          ++p;
        }
        if (++s == OZ_STAGES) {
          s = 0;
          ph ^= 1u;
        }
      }
      if (g >= 0 && ok) umma_commit(&acc_full[g & 1]);
      // every MMA of this thread has completed before tensor memory is released
      umma_commit(done);
      if (!mbar_wait(done, 0)) ok = false;
    }
  } else {
    // epilogue warps: warp w owns accumulator lanes (output rows) 32 (w % 4) .. + 31 and the 64
    // columns starting at 64 (w / 4)
    const int quarter = warp & 3, ch = 64 * (warp >> 2);
    int G = 0;
    {
      int gt = 0, prev = -1, p = s0 / nk, kt = s0 - p * nk;
      for (int n = s0; n < s1; ++n) {
        const int lv = P.lv[p];
        if (oz_new_group(prev, lv, gt)) {
          ++G;
          gt = 0;
        }
        ++gt;
        prev = lv;
        if (++kt == nk) {
          kt = 0;
          ++p;
        }
      }
    }
    float hi[64], lo[64];
#pragma unroll
    for (int j = 0; j < 64; ++j) hi[j] = lo[j] = 0.0f;
    for (int g = 0; g < G; ++g) {
      if (!mbar_wait(&acc_full[g & 1], ((uint32_t)g >> 1) & 1u)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t base = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)((g & 1) * OZ_BN + ch);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        uint32_t r[32];
        tmem_ld_32cols(base + 32 * h, r);
#pragma unroll
        for (int j = 0; j < 32; ++j) ff_add(hi[32 * h + j], lo[32 * h + j], __uint_as_float(r[j]));
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[g & 1]);
    }
    if (ok) {
      // Every MMA has completed (the last group's commit covers them), so the operand ring is
      // free: each warp stages its 32 x 64 (hi, lo) block there and writes it back row by row,
      // 32 consecutive columns per store instruction.
      float2* buf = (float2*)(smem + (size_t)warp * 32 * 65 * sizeof(float2));
#pragma unroll
      for (int j = 0; j < 64; ++j) buf[lane * 65 + j] = make_float2(hi[j], lo[j]);
      __syncwarp();
      const int rbase = m0 + quarter * 32;
      for (int rr = 0; rr < 32; ++rr) {
        const int row = rbase + rr;
        if (row >= P.M) break;
        float2* wr = P.W + ((size_t)z * P.M + row) * P.N;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int col = n0 + ch + 32 * h + lane;
          if (col < P.N) wr[col] = buf[rr * 65 + 32 * h + lane];
        }
      }
    }
  }
  if (!ok) atomicExch(P.err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, Cfg::TMEM_COLS);
}

// ------------------------------------------------------------------ slicing
// Logical operand: element (r, k) = (trans ? src[k ld + r] : src[r ld + k]) * (scale ? scale[k] : 1)
// for r < rows, k < K.
struct OzOperand {
  int rows, K;
  const double* src;
  int ld, trans;
  const double* scale;
  int* part;                 // ceil(K / 64) x rows exponent partials
  __nv_bfloat16* out;        // rows x (s * Kp)
  double* fac;               // rows: mult * 2^(e_r - 7)
  double mult;
};
struct OzSplitArgs {
  OzOperand op[2];
  int Kp, s;
};

__device__ __forceinline__ int biased_exp(double v) { return oz::biased_exp(v); }

__device__ __forceinline__ double oz_load(const OzOperand& o, int r, int k) {
  double v = o.trans ? o.src[(size_t)k * o.ld + r] : o.src[(size_t)r * o.ld + k];
  if (o.scale) v *= o.scale[k];
  return v;
}

// part[kb][r] = max biased exponent of v(r, k) over the 64 k of block kb
__global__ void k_oz_rowexp(OzSplitArgs a) {
  const OzOperand& o = a.op[blockIdx.z];
  const int r0 = blockIdx.y * 32, k0 = blockIdx.x * 64;
  if (r0 >= o.rows || k0 >= o.K) return;
  const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
  if (o.trans) {
    __shared__ int sm[8][33];
    const int r = r0 + tx;
    int e = 0;
    if (r < o.rows)
      for (int kk = ty; kk < 64; kk += 8) {
        const int k = k0 + kk;
        if (k < o.K) e = max(e, biased_exp(oz_load(o, r, k)));
      }
    sm[ty][tx] = e;
    __syncthreads();
    if (ty == 0 && r < o.rows) {
#pragma unroll
      for (int y = 1; y < 8; ++y) e = max(e, sm[y][tx]);
      o.part[(size_t)blockIdx.x * o.rows + r] = e;
    }
  } else {
    for (int i = ty; i < 32; i += 8) {
      const int r = r0 + i;
      int e = 0;
      if (r < o.rows)
        for (int kk = tx; kk < 64; kk += 32) {
          const int k = k0 + kk;
          if (k < o.K) e = max(e, biased_exp(oz_load(o, r, k)));
        }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, off));
      if (tx == 0 && r < o.rows) o.part[(size_t)blockIdx.x * o.rows + r] = e;
    }
  }
}

__device__ __forceinline__ void oz_digits(double v, int er, int s, int (&d)[OZ_MAX_SLICES]) {
  oz::digits(v, er, s, d);
}

// Slicing for K > kOzClusterK: row exponents from the partials of k_oz_rowexp.
__global__ void k_oz_split(OzSplitArgs a) {
  const OzOperand& o = a.op[blockIdx.z];
  const int r0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
  if (r0 >= o.rows) return;
  const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
  const int s = a.s, Kp = a.Kp;
  __shared__ double tile[32][33];
  __shared__ int se[32];
  if (ty == 0) {
    const int r = r0 + tx;
    int E = 0;
    if (r < o.rows) {
      const int nkb = (o.K + 63) / 64;
      for (int kb = 0; kb < nkb; ++kb) E = max(E, o.part[(size_t)kb * o.rows + r]);
    }
    if (blockIdx.x == 0 && r < o.rows)
      o.fac[r] = (E == 0x7FF) ? __longlong_as_double(0x7FF8000000000000ll) : ldexp(o.mult, E - 1022 - 7);
    se[tx] = E - 1022;   // row exponent e_r
  }
  for (int i = ty; i < 32; i += 8) {
    if (o.trans) {
      const int k = k0 + i, r = r0 + tx;
      tile[tx][i] = (k < o.K && r < o.rows) ? o.src[(size_t)k * o.ld + r] : 0.0;
    } else {
      const int r = r0 + i, k = k0 + tx;
      tile[i][tx] = (k < o.K && r < o.rows) ? o.src[(size_t)r * o.ld + k] : 0.0;
    }
  }
  __syncthreads();
  const size_t rowlen = (size_t)s * Kp;
  for (int i = ty; i < 32; i += 8) {
    const int r = r0 + i, k = k0 + tx;
    if (r >= o.rows || k >= Kp) continue;
    double v = tile[i][tx];
    if (o.scale && k < o.K) v *= o.scale[k];
    int d[OZ_MAX_SLICES];
    oz_digits(v, se[i], s, d);
    __nv_bfloat16* dst = o.out + (size_t)r * rowlen + k;
#pragma unroll
    for (int j = 0; j < OZ_MAX_SLICES; ++j) {
      if (j < s) {
        // d_j 2^(-8 j): at most 8 significant bits, so the BF16 truncation is exact
        const float f = __int2float_rn(d[j]) * __int_as_float((127 - 8 * j) << 23);
        dst[(size_t)j * Kp] = __ushort_as_bfloat16((unsigned short)(__float_as_uint(f) >> 16));
      }
    }
  }
}

// Slicing for K <= kOzClusterK in one launch: a cluster of at most 8 CTAs spans the K range of
// 32 logical rows, each CTA 64 KW columns.  Each CTA keeps its values in shared memory, publishes
// its per-row maximum exponents, reads its peers' through distributed shared memory, and slices
// its own values (no second pass over the operand, no second launch).  All CTAs of a cluster
// share blockIdx.y and blockIdx.z, so a cluster is either wholly inside the operand or outside.
template <int KW>
__global__ void __launch_bounds__(32 * kSplitRows) k_oz_split_cluster(OzSplitArgs a) {
  constexpr int COLS = 64 * KW;
  pdl_wait();
  pdl_trigger();
  cg::cluster_group cluster = cg::this_cluster();
  const OzOperand& o = a.op[blockIdx.z];
  const int r0 = blockIdx.y * 32, k0 = blockIdx.x * COLS;
  if (r0 >= o.rows) return;
  const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x kSplitRows
  const int s = a.s, Kp = a.Kp;
  extern __shared__ double tile_raw[];            // [32][COLS + 1]
  double (*tile)[COLS + 1] = reinterpret_cast<double (*)[COLS + 1]>(tile_raw);
  __shared__ int pmax[32], se[32];
  if (o.trans) {
    const int r = r0 + tx;
#pragma unroll
    for (int kk = ty; kk < COLS; kk += kSplitRows) {
      const int k = k0 + kk;
      tile[tx][kk] = (k < o.K && r < o.rows) ? oz_load(o, r, k) : 0.0;
    }
  } else {
#pragma unroll
    for (int i = ty; i < 32; i += kSplitRows) {
      const int r = r0 + i;
#pragma unroll
      for (int h = 0; h < 2 * KW; ++h) {
        const int k = k0 + tx + 32 * h;
        tile[i][tx + 32 * h] = (k < o.K && r < o.rows) ? oz_load(o, r, k) : 0.0;
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = ty; i < 32; i += kSplitRows) {
    int e = 0;
#pragma unroll
    for (int h = 0; h < 2 * KW; ++h) e = max(e, biased_exp(tile[i][tx + 32 * h]));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, off));
    if (tx == 0) pmax[i] = e;
  }
  cluster.sync();
  if (ty == 0) {
    int E = 0;
    for (unsigned q = 0; q < cluster.num_blocks(); ++q) E = max(E, cluster.map_shared_rank(pmax, q)[tx]);
    const int r = r0 + tx;
    if (blockIdx.x == 0 && r < o.rows)
      o.fac[r] = (E == 0x7FF) ? __longlong_as_double(0x7FF8000000000000ll) : ldexp(o.mult, E - 1022 - 7);
    se[tx] = E - 1022;
  }
  cluster.sync();   // peers are done reading pmax; se is visible block-wide
  const size_t rowlen = (size_t)s * Kp;
#pragma unroll
  for (int i = ty; i < 32; i += kSplitRows) {
    const int r = r0 + i;
    if (r >= o.rows) continue;
#pragma unroll
    for (int h = 0; h < 2 * KW; ++h) {
      const int k = k0 + tx + 32 * h;
      if (k >= Kp) continue;
      int d[OZ_MAX_SLICES];
      oz_digits(tile[i][tx + 32 * h], se[i], s, d);
      __nv_bfloat16* dst = o.out + (size_t)r * rowlen + k;
#pragma unroll
      for (int j = 0; j < OZ_MAX_SLICES; ++j)
        if (j < s) {
          const float f = __int2float_rn(d[j]) * __int_as_float((127 - 8 * j) << 23);
          dst[(size_t)j * Kp] = __ushort_as_bfloat16((unsigned short)(__float_as_uint(f) >> 16));
        }
    }
  }
}

template <int KW>
void launch_split_cluster(cudaStream_t st, const OzSplitArgs& sa, int Kp, int rb) {
  const int ncta = (Kp + 64 * KW - 1) / (64 * KW);
  const size_t smem = (size_t)32 * (64 * KW + 1) * sizeof(double);
  static bool attr[64] = {};   // the attribute is per device
  const int dev = device_index();
  if (!attr[dev]) {
    KOT_CUDA(cudaFuncSetAttribute(k_oz_split_cluster<KW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr[dev] = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ncta, rb, 2);
  cfg.blockDim = dim3(32, kSplitRows);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attrs[2];
  attrs[0].id = cudaLaunchAttributeClusterDimension;
  attrs[0].val.clusterDim.x = (unsigned)ncta;
  attrs[0].val.clusterDim.y = 1;
  attrs[0].val.clusterDim.z = 1;
  attrs[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;   // see launch_pdl
  attrs[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attrs;
  cfg.numAttrs = pdl_enabled() ? 2 : 1;
  KOT_CUDA(cudaLaunchKernelEx(&cfg, k_oz_split_cluster<KW>, sa));
}

// ------------------------------------------------------------------ finalize
__device__ __forceinline__ double oz_value(const float2* __restrict__ W, size_t MN, int splits, size_t idx) {
  float2 u[OZ_MAX_SPLITS];
#pragma unroll
  for (int z = 0; z < OZ_MAX_SPLITS; ++z)
    if (z < splits) u[z] = __ldcs(W + (size_t)z * MN + idx);   // all loads in flight at once
  float hi = u[0].x, lo = u[0].y;
#pragma unroll
  for (int z = 1; z < OZ_MAX_SPLITS; ++z)
    if (z < splits) {
      ff_add(hi, lo, u[z].x);
      lo = __fadd_rn(lo, u[z].y);
    }
  return (double)hi + (double)lo;
}

__global__ void k_oz_finalize(int M, int N, int splits, const float2* __restrict__ W,
                              const double* __restrict__ fa, const double* __restrict__ fb, double beta,
                              double* __restrict__ C, int ldc, int sym) {
  pdl_wait();
  pdl_trigger();
  const size_t MN = (size_t)M * N;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < MN;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx / N), c = (int)(idx - (size_t)r * N);
    if (sym && c < r) continue;   // a symmetric result: entries on or above the diagonal, mirrored
    const double v = oz_value(W, MN, splits, idx) * fa[r] * fb[c];
    if (sym && c != r) {
      double* cm = C + (size_t)c * ldc + r;
      *cm = (beta == 0.0) ? v : fma(beta, *cm, v);
    }
    double* cp = C + (size_t)r * ldc + c;
    *cp = (beta == 0.0) ? v : fma(beta, *cp, v);
  }
}

}  // namespace

namespace {
template <int BN>
void launch_oz_gemm(cudaStream_t st, const CUtensorMap& ta, const CUtensorMap& tb, const OzPlan& P, int M, int N,
                    int splits) {
  using Cfg = OzCfg<BN>;
  static bool attr_set[64] = {};   // the attribute is per device
  const int dev = device_index();
  if (!attr_set[dev]) {
    KOT_CUDA(cudaFuncSetAttribute(k_oz_gemm<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM));
    attr_set[dev] = true;
  }
  launch_pdl(k_oz_gemm<BN>, dim3(cdiv(N, BN), cdiv(M, OZ_BM), splits), dim3(Cfg::THREADS), Cfg::SMEM, st,
             ta, tb, P);
}
}  // namespace

void gemm_oz(cudaStream_t st, OzWork& w, int M, int N, int K, const TcOperand& A, const TcOperand& B,
             int slices, double alpha, double beta, double* C, int ldc, bool sym) {
  if (M <= 0 || N <= 0) return;
  if (slices < 3 || slices > OZ_MAX_SLICES) throw Error{KOT_ERR_INVALID, "gemm_oz: slices must be 3..8"};
  if (sym && M != N) throw Error{KOT_ERR_INVALID, "gemm_oz: a symmetric result needs M == N"};
  if (K <= 0) {
    if (beta == 0.0)
      for (int i = 0; i < M; ++i) KOT_CUDA(cudaMemsetAsync(C + (size_t)i * ldc, 0, N * sizeof(double), st));
    return;
  }
  const int s = slices;
  const int Kp = cdiv(K, OZ_BK) * OZ_BK;
  const int nkb = cdiv(K, 64);
  const int nsm = sm_count();

  OzPlan P;
  P.M = M;
  P.N = N;
  P.Kp = Kp;
  P.nk = Kp / OZ_BK;
  int np = 0;
  for (int t = 0; t < s; ++t)
    for (int i = 0; i <= t; ++i) {
      P.pa[np] = (signed char)i;
      P.pb[np] = (signed char)(t - i);
      P.lv[np] = (signed char)t;
      ++np;
    }
  P.npairs = np;
  // wide tiles from 256 up (twice the MMA work per 64-wide K step for 1.33x the bytes, and fewer,
  // longer CTAs: inside the solve at l = 300, where the EG lane and the Newton step share the GPU,
  // 128-wide tiles ran 4% faster than 64-wide ones), unless the autotuner chose for this size
  // bucket; w.bn_override (the tuner's probe) wins
  int BNsel = (M >= 256 && N >= 256) ? 128 : 64;
  const int tuned_bn = tuned_tile_width(device_index(), std::max(M, N), s);
  if (tuned_bn == 64 || tuned_bn == 128) BNsel = tuned_bn;
  if (w.bn_override == 64 || w.bn_override == 128) BNsel = w.bn_override;
  const int tiles = cdiv(N, BNsel) * cdiv(M, OZ_BM);
  // split count: the autotuner's choice for this size bucket and slice count if there is one,
  // else enough splits to give every SM a CTA (at most kOzDefaultSplits, which measured best in
  // the solve at l = 300); w.splits_override (the tuner's probe) wins
  int want = std::max(1, std::min(kOzDefaultSplits, nsm / tiles));
  const int tuned = tuned_splits(device_index(), std::max(M, N), s);
  if (tuned > 0) want = tuned;
  if (w.splits_override > 0) want = w.splits_override;
  const int splits = std::max(1, std::min({OZ_MAX_SPLITS, np * (Kp / OZ_BK), want}));
  const int T = np * P.nk;   // tile steps (pair, k tile) of one output tile
  for (int z = 0; z <= splits; ++z) P.sbeg[z] = (int)((long long)z * T / splits);

  w.a.alloc((size_t)M * s * Kp);
  w.b.alloc((size_t)N * s * Kp);
  w.part.alloc((size_t)nkb * (M + N));
  w.fac.alloc((size_t)M + N);
  w.w.alloc((size_t)splits * M * N);
  if (!w.err.p) {
    w.err.alloc(1);
    KOT_CUDA(cudaMemsetAsync(w.err.p, 0, sizeof(int), st));
  }
  P.W = w.w.p;
  P.err = w.err.p;
  P.sym = sym ? 1 : 0;

  OzSplitArgs sa;
  sa.Kp = Kp;
  sa.s = s;
  const TcOperand* ops[2] = {&A, &B};
  const int rows[2] = {M, N};
  for (int q = 0; q < 2; ++q) {
    OzOperand& o = sa.op[q];
    o.rows = rows[q];
    o.K = K;
    o.src = ops[q]->src;
    o.ld = ops[q]->ld;
    o.trans = ops[q]->trans ? 1 : 0;
    o.scale = ops[q]->scale;
    o.part = w.part.p + (q == 0 ? 0 : (size_t)nkb * M);
    o.out = (__nv_bfloat16*)(q == 0 ? w.a.p : w.b.p);
    o.fac = w.fac.p + (q == 0 ? 0 : M);
    o.mult = q == 0 ? alpha : 1.0;
  }
  const int rb = cdiv(std::max(M, N), 32);
  const dim3 bs(32, 8);
  {
    // bytes: FP64 operands read twice, BF16 slices written
    ProfScope ps(st, KC_OZ_AUX, 0.0, 16.0 * ((double)M + N) * K + 2.0 * s * ((double)M + N) * Kp);
    if (K <= kOzClusterK) {
      // widest CTA that keeps the cluster at <= 8 CTAs
      if (Kp <= 8 * 64) launch_split_cluster<1>(st, sa, Kp, rb);
      else if (Kp <= 8 * 128) launch_split_cluster<2>(st, sa, Kp, rb);
      else launch_split_cluster<4>(st, sa, Kp, rb);
      KOT_LAUNCHED(1);
    } else {
      k_oz_rowexp<<<dim3(nkb, rb, 2), bs, 0, st>>>(sa);
      k_oz_split<<<dim3(Kp / 32, rb, 2), bs, 0, st>>>(sa);
      KOT_LAUNCHED(2);
    }
  }

  // descriptors are re-encoded only when the slice buffers or their shapes change
  if (w.key_a != w.a.p || w.rows_a != M || w.cols_a != s * Kp) {
    const CUtensorMap m = make_bf16_map(w.a.p, M, s * Kp, OZ_BM);
    std::memcpy(w.map_a, &m, sizeof(m));
    w.key_a = w.a.p;
    w.rows_a = M;
    w.cols_a = s * Kp;
  }
  if (w.key_b != w.b.p || w.rows_b != N || w.cols_b != s * Kp || w.box_b != BNsel) {
    const CUtensorMap m = make_bf16_map(w.b.p, N, s * Kp, BNsel);
    std::memcpy(w.map_b, &m, sizeof(m));
    w.key_b = w.b.p;
    w.rows_b = N;
    w.cols_b = s * Kp;
    w.box_b = BNsel;
  }
  CUtensorMap ta, tb;
  std::memcpy(&ta, w.map_a, sizeof(ta));
  std::memcpy(&tb, w.map_b, sizeof(tb));
  {
    // algorithmic work: the product it stands for, 2 M N K flops; executed: np BF16 slice-pair
    // products of 2 M N K flops each; bytes: the BF16 slices in, the float2 partial sums out
    ProfScope ps(st, KC_GEMM_OZ, 2.0 * M * N * (double)K,
                 2.0 * s * ((double)M + N) * Kp + 8.0 * splits * (double)M * N, 2.0 * M * N * (double)K * np);
    if (BNsel == 128) launch_oz_gemm<128>(st, ta, tb, P, M, N, splits);
    else launch_oz_gemm<64>(st, ta, tb, P, M, N, splits);
    KOT_LAUNCHED(1);
  }
  const size_t MN = (size_t)M * N;
  const int fgrid = (int)std::min<size_t>(cdiv(MN, 256), (size_t)nsm * 8);
  {
    ProfScope ps(st, KC_OZ_AUX, 0.0, 8.0 * splits * (double)MN + 8.0 * (beta == 0.0 ? 1.0 : 2.0) * (double)MN);
    launch_pdl(k_oz_finalize, dim3(fgrid), dim3(256), 0, st, M, N, splits, (const float2*)w.w.p,
               (const double*)w.fac.p, (const double*)(w.fac.p + M), beta, C, ldc, sym ? 1 : 0);
    KOT_LAUNCHED(1);
  }
}

int tuned_splits(int dev, int mn, int slices) {
  if (dev < 0 || dev >= 64 || slices < 0 || slices > OZ_MAX_SLICES) return 0;
  return g_tuned_splits[dev][size_bucket(mn)][slices];
}

void set_tuned_splits(int dev, int mn, int slices, int splits) {
  if (dev < 0 || dev >= 64 || slices < 0 || slices > OZ_MAX_SLICES) return;
  g_tuned_splits[dev][size_bucket(mn)][slices] = std::max(0, std::min(splits, OZ_MAX_SPLITS));
}

int tuned_tile_width(int dev, int mn, int slices) {
  if (dev < 0 || dev >= 64 || slices < 0 || slices > OZ_MAX_SLICES) return 0;
  return g_tuned_bn[dev][size_bucket(mn)][slices];
}

void set_tuned_tile_width(int dev, int mn, int slices, int bn) {
  if (dev < 0 || dev >= 64 || slices < 0 || slices > OZ_MAX_SLICES) return;
  g_tuned_bn[dev][size_bucket(mn)][slices] = (bn == 64 || bn == 128) ? bn : 0;
}

int gemm_oz_error(cudaStream_t st, OzWork& w) {
  if (!w.err.p) return 0;
  int h = 0;
  KOT_CUDA(cudaMemcpyAsync(&h, w.err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  KOT_CUDA(cudaStreamSynchronize(st));
  if (h) KOT_CUDA(cudaMemsetAsync(w.err.p, 0, sizeof(int), st));
  return h;
}

void gemm_acc(cudaStream_t st, OzWork* oz, bool ta, bool tb, int M, int N, int K, double alpha,
              const double* A, int lda, const double* B, int ldb, const double* s, double beta,
              double* C, int ldc, int flags) {
  const double work = 2.0 * M * N * K * ((flags & G_SYM) ? 0.5 : 1.0);
  if (!oz || work < oz->f64_below)
    return gemm_f64(st, ta, tb, M, N, K, alpha, A, lda, B, ldb, s, beta, C, ldc, flags);
  // gemm_f64's op(B) is K x N; the tensor-core form takes it as N rows of K
  gemm_oz(st, *oz, M, N, K, TcOperand{A, lda, ta, s}, TcOperand{B, ldb, !tb, nullptr}, oz->slices, alpha,
          beta, C, ldc, (flags & G_SYM) != 0);
}

}  // namespace kot
