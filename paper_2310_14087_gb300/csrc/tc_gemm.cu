// Dense products on the 5th-generation tensor cores: C = alpha * opA(A) * opB(B)^T + beta * C
// with FP64 inputs and outputs and BF16 x BF16 -> FP32 tensor-core arithmetic.
//
// Precision: each FP64 operand value v is split into up to three BF16 pieces v ~ p0 + p1 + p2
// (8 significant bits each).  The product sum_{i+j<pieces} A_i B_j^T is formed in ONE
// accumulation by laying the pieces out as consecutive K-segments of the operands
// ([A0 A0 A0 A1 A1 A2] times [B0 B1 B2 B0 B1 B0]^T for three pieces), so the GEMM kernel itself
// is a plain BF16 GEMM with FP32 accumulation in tensor memory.  One piece gives BF16 accuracy
// (~4e-3 relative), three give ~FP32 accuracy (~1e-7 relative per term).
//
// Kernel: one CTA per 128 x 128 output tile, 4 warps.  Warp 0 lane 0 streams 128 x 64 BF16
// tiles of both operands into a 4-stage shared-memory ring with TMA (128-byte swizzle, mbarrier
// completion); warp 1 lane 0 issues tcgen05.mma (M = 128, N = 128, K = 16 per instruction) into
// a 128-column FP32 accumulator in tensor memory and releases each stage with tcgen05.commit; all
// four warps then read their 32 accumulator lanes with tcgen05.ld and write FP64 results.
// Every mbarrier wait is bounded: on timeout the CTA records an error flag, still frees its
// tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "kot_internal.cuh"
#include "tc_ptx.cuh"

namespace kot {

namespace {

constexpr int TC_BM = 128, TC_BN = 128, TC_BK = 64, TC_STAGES = 4, TC_THREADS = 128;
constexpr int TILE_A_BYTES = TC_BM * TC_BK * 2;   // 16 KB
constexpr int TILE_B_BYTES = TC_BN * TC_BK * 2;   // 16 KB
constexpr int STAGE_BYTES = TILE_A_BYTES + TILE_B_BYTES;
constexpr int TC_SMEM = TC_STAGES * STAGE_BYTES + 1024 + 256;
constexpr int TMEM_COLS = 128;

inline int cdiv(size_t a, int b) { return (int)((a + b - 1) / b); }

__global__ void __launch_bounds__(TC_THREADS, 1)
    k_tc_gemm_bf16(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
                   double* __restrict__ C, int M, int N, int Ktot, int ldc, double alpha,
                   double beta, int* __restrict__ err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + TC_STAGES * STAGE_BYTES);
  uint64_t* empty = full + TC_STAGES;
  uint64_t* done = empty + TC_STAGES;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * TC_BM, n0 = blockIdx.x * TC_BN;
  const int nk = Ktot / TC_BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  bool ok = true;

  if (warp == 0 && lane == 0) {
    // TMA producer
    for (int kt = 0; kt < nk; ++kt) {
      const int s = kt % TC_STAGES;
      const uint32_t ph = (uint32_t)(kt / TC_STAGES) & 1u;
      if (!mbar_wait(&empty[s], ph ^ 1u)) {
        ok = false;
        break;
      }
      mbar_expect_tx(&full[s], STAGE_BYTES);
      uint8_t* st = smem + s * STAGE_BYTES;
      tma_load_2d(st, &ta, &full[s], kt * TC_BK, m0);
      tma_load_2d(st + TILE_A_BYTES, &tb, &full[s], kt * TC_BK, n0);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    constexpr uint32_t idesc = idesc_bf16(TC_BM, TC_BN);
    for (int kt = 0; kt < nk; ++kt) {
      const int s = kt % TC_STAGES;
      const uint32_t ph = (uint32_t)(kt / TC_STAGES) & 1u;
      if (!mbar_wait(&full[s], ph)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a_addr = smem_u32(smem + s * STAGE_BYTES);
      const uint32_t b_addr = a_addr + TILE_A_BYTES;
#pragma unroll
      for (int k = 0; k < TC_BK / 16; ++k)
        umma_bf16(tmem, smem_desc_sw128(a_addr + 32 * k), smem_desc_sw128(b_addr + 32 * k), idesc,
                  (kt > 0 || k > 0) ? 1u : 0u);
      umma_commit(&empty[s]);
    }
    umma_commit(done);
  }
  __syncwarp();
  // epilogue: warp w owns accumulator lanes (rows) 32 w .. 32 w + 31
  if (!mbar_wait(done, 0)) ok = false;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int row = m0 + warp * 32 + lane;
#pragma unroll 1
  for (int c0 = 0; c0 < TC_BN; c0 += 32) {
    uint32_t r[32];
    tmem_ld_32cols(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
    if (row < M && ok) {
      double* crow = C + (size_t)row * ldc;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int col = n0 + c0 + j;
        if (col < N) {
          const double v = alpha * (double)__uint_as_float(r[j]);
          crow[col] = (beta == 0.0) ? v : fma(beta, crow[col], v);
        }
      }
    }
  }
  if (!ok) atomicExch(err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS)
                 : "memory");
}

// out[r][s*Kp + k] = piece_{code(s)}(v(r, k)), v(r, k) = (trans ? src[k][r] : src[r][k]) * scale[k]
// (0 for k >= K).  The three pieces: p0 = bf16(v), p1 = bf16(v - p0), p2 = bf16(v - p0 - p1).
__global__ void k_split_bf16(int rows, int K, int Kp, int nseg, unsigned codes,
                             const double* __restrict__ src, int ld, int trans,
                             const double* __restrict__ scale, __nv_bfloat16* __restrict__ out) {
  __shared__ double tile[32][33];
  const int k0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
  // stage a 32 x 32 block of v with coalesced reads in either orientation
  for (int i = ty; i < 32; i += 8) {
    if (trans) {
      const int k = k0 + i, r = r0 + tx;
      tile[tx][i] = (k < K && r < rows) ? src[(size_t)k * ld + r] : 0.0;
    } else {
      const int r = r0 + i, k = k0 + tx;
      tile[i][tx] = (k < K && r < rows) ? src[(size_t)r * ld + k] : 0.0;
    }
  }
  __syncthreads();
  const size_t rowlen = (size_t)nseg * Kp;
  for (int i = ty; i < 32; i += 8) {
    const int r = r0 + i, k = k0 + tx;
    if (r >= rows || k >= Kp) continue;
    double v = tile[i][tx];
    if (scale && k < K) v *= scale[k];
    const __nv_bfloat16 p0 = __float2bfloat16_rn((float)v);
    const double rem1 = v - (double)__bfloat162float(p0);
    const __nv_bfloat16 p1 = __float2bfloat16_rn((float)rem1);
    const double rem2 = rem1 - (double)__bfloat162float(p1);
    const __nv_bfloat16 p2 = __float2bfloat16_rn((float)rem2);
    for (int s = 0; s < nseg; ++s) {
      const unsigned c = (codes >> (2 * s)) & 3u;
      out[(size_t)r * rowlen + (size_t)s * Kp + k] = (c == 0) ? p0 : (c == 1 ? p1 : p2);
    }
  }
}


PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  std::call_once(g_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  });
  if (!g_encode) throw Error{KOT_ERR_CUDA, "cuTensorMapEncodeTiled is not available"};
  return g_encode;
}

}  // namespace

CUtensorMap make_bf16_map(const void* base, int rows, int cols, int box_rows) {
  CUtensorMap m;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encoder()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides,
                         box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Error{KOT_ERR_CUDA, "cuTensorMapEncodeTiled failed"};
  return m;
}

namespace {

// Segment codes: the (i, j) piece pairs with i + j < pieces, A gets i and B gets j.
void segment_codes(int pieces, unsigned* ca, unsigned* cb, int* nseg) {
  unsigned a = 0, b = 0;
  int s = 0;
  for (int i = 0; i < pieces; ++i)
    for (int j = 0; i + j < pieces; ++j) {
      a |= (unsigned)i << (2 * s);
      b |= (unsigned)j << (2 * s);
      ++s;
    }
  *ca = a;
  *cb = b;
  *nseg = s;
}

}  // namespace

void gemm_tc(cudaStream_t st, TcWork& w, int M, int N, int K, const TcOperand& A,
             const TcOperand& B, int pieces, double alpha, double beta, double* C, int ldc) {
  if (M <= 0 || N <= 0) return;
  if (pieces < 1 || pieces > 3) throw Error{KOT_ERR_INVALID, "gemm_tc: pieces must be 1..3"};
  const int Kp = std::max(TC_BK, cdiv(std::max(K, 1), TC_BK) * TC_BK);
  unsigned ca, cb;
  int nseg;
  segment_codes(pieces, &ca, &cb, &nseg);
  const int Ktot = nseg * Kp;
  w.a.alloc((size_t)M * Ktot);
  w.b.alloc((size_t)N * Ktot);
  if (!w.err.p) {
    w.err.alloc(1);
    KOT_CUDA(cudaMemsetAsync(w.err.p, 0, sizeof(int), st));
  }
  dim3 bs(32, 8);
  k_split_bf16<<<dim3(cdiv(Kp, 32), cdiv(M, 32)), bs, 0, st>>>(M, K, Kp, nseg, ca, A.src, A.ld, A.trans ? 1 : 0,
                                                             A.scale, (__nv_bfloat16*)w.a.p);
  k_split_bf16<<<dim3(cdiv(Kp, 32), cdiv(N, 32)), bs, 0, st>>>(N, K, Kp, nseg, cb, B.src, B.ld, B.trans ? 1 : 0,
                                                             B.scale, (__nv_bfloat16*)w.b.p);
  KOT_LAUNCHED(2);
  const CUtensorMap ta = make_bf16_map(w.a.p, M, Ktot, TC_BM);
  const CUtensorMap tb = make_bf16_map(w.b.p, N, Ktot, TC_BN);
  static bool attr_set[64] = {};   // the attribute is per device
  int adev = 0;
  KOT_CUDA(cudaGetDevice(&adev));
  if (adev < 0 || adev >= 64) throw Error{KOT_ERR_CUDA, "device ordinal out of range"};
  if (!attr_set[adev]) {
    KOT_CUDA(cudaFuncSetAttribute(k_tc_gemm_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
    attr_set[adev] = true;
  }
  ProfScope ps(st, KC_GEMM_TC, 2.0 * M * N * (double)K * nseg, 2.0 * ((double)M + N) * Ktot + 8.0 * M * N);
  k_tc_gemm_bf16<<<dim3(cdiv(N, TC_BN), cdiv(M, TC_BM)), TC_THREADS, TC_SMEM, st>>>(ta, tb, C, M, N, Ktot, ldc,
                                                                               alpha, beta, w.err.p);
  KOT_LAUNCHED(1);
}

namespace {
// Failure-detection probe: one thread waits, with the same bounded poll as the tensor-core
// kernels, on an mbarrier that expects one arrival nobody makes; when the polls run out it records
// the timeout in *err, exactly as a starved pipeline stage would, and the kernel returns.
__global__ void k_starved_wait(long long polls, int* __restrict__ err) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  for (long long i = 0; i < polls; ++i) {
    if (mbar_try_wait(&bar, 0)) return;   // never: nothing arrives
    __nanosleep(20);
  }
  atomicExch(err, 1);
}
}  // namespace

int starved_wait_probe(cudaStream_t st, TcWork& w, long long polls) {
  if (!w.err.p) {
    w.err.alloc(1);
    KOT_CUDA(cudaMemsetAsync(w.err.p, 0, sizeof(int), st));
  }
  k_starved_wait<<<1, 32, 0, st>>>(polls, w.err.p);
  KOT_CHECK_LAUNCH();
  return gemm_tc_error(st, w);
}

int gemm_tc_error(cudaStream_t st, TcWork& w) {
  if (!w.err.p) return 0;
  int h = 0;
  KOT_CUDA(cudaMemcpyAsync(&h, w.err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  KOT_CUDA(cudaStreamSynchronize(st));
  if (h) KOT_CUDA(cudaMemsetAsync(w.err.p, 0, sizeof(int), st));
  return h;
}

}  // namespace kot
