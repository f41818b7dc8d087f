// Tensor-core local products Z_p = S_p^+ Y_p on sm_103a: tcgen05.mma (kind::tf32, or kind::f16 with bf16
// operands) with the accumulators in TMEM, operands staged by TMA (64-byte swizzle) through a 3-stage mbarrier
// pipeline.
//
// Precision: both operands are split into pairs, x = hi + lo with hi = round(x) to the operand type and
// lo = x - hi rounded again, and the product is taken as hi*hi + hi*lo + lo*hi (three MMAs into one FP32
// accumulator).  tf32 pairs carry ~22 significant bits (relative error near 2^-21 per product, close to FP32
// local products); bf16 pairs carry 16 (near 2^-16, at twice the tensor rate of tf32).  The FP64 outer
// refinement of the solver removes either error.
//
// One CTA computes a 256 (rows of S^+) x 256 (right-hand sides) tile of one pattern as two 128 x 256 halves,
// each an MMA of M = 128, N = 256 into its own TMEM accumulator (the two fill the 512 TMEM columns): both halves
// use the same staged right-hand-side tile, so a K step loads 64 KB for 12 MMAs instead of 96 KB for 12 with one
// 128-row half (operand bytes per flop from L2 are what limits this kernel).  Warp roles: warp 0 lane 0 issues
// TMA loads, warp 1 lane 0 issues the MMAs, all eight warps drain TMEM in the epilogue (warps w and w + 4 the
// same 32 TMEM lanes of the two halves).  Every wait on an mbarrier is bounded: on expiry the CTA records an
// error code, stops issuing work, waits (again bounded) for its own MMAs to retire, frees TMEM and returns.
#include <cuda.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "ops.cuh"
#include "tc.cuh"

namespace fetirp {

namespace {

// 256 x 256 output tile per CTA (two 128 x 256 halves)
constexpr int BM = 256, BMH = 128, BN = 256;
constexpr int ROW_BYTES = 64;                     // one K step of a tile row = one 64-byte swizzle row
constexpr int STAGES = 3;
constexpr int TILE_A_BYTES = BM * ROW_BYTES;      // 16 KB (both halves; the second starts 8 KB in)
constexpr int TILE_B_BYTES = BN * ROW_BYTES;      // 16 KB
constexpr int STAGE_BYTES = 2 * TILE_A_BYTES + 2 * TILE_B_BYTES;   // A_hi, A_lo, B_hi, B_lo: 64 KB
constexpr int TMEM_COLS = 2 * BN;                 // two FP32 accumulators of 256 columns
constexpr int THREADS = 256;
// stages, 1024 bytes of alignment slack, barriers and flags, and 4 KB of margin past the last stage
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256 + 4096;
constexpr unsigned long long WAIT_NS = 2000000000ull;  // a bounded wait gives up after 2 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait; returns false on expiry.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = now_ns();
  while (now_ns() - t0 < WAIT_NS)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void tma_load_2d(const CUtensorMap* map, uint64_t* bar, void* dst, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// Shared-memory matrix descriptor (tcgen05): K-major, 64-byte swizzle, 8-row groups 512 bytes apart.
__device__ __forceinline__ uint64_t smem_desc(const void* p) {
  const uint64_t addr = smem_u32(p);
  uint64_t d = 0;
  d |= (addr >> 4) & 0x3FFFull;                 // start address
  d |= (uint64_t)(16 >> 4) << 16;               // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)((8 * ROW_BYTES) >> 4) << 32;  // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;                       // descriptor version (sm_100 family)
  d |= (uint64_t)4 << 61;                       // layout: SWIZZLE_64B
  return d;
}

// Instruction descriptor: D f32, A/B tf32 (kind::tf32) or bf16 (kind::f16), both K-major, N = BN, M = BM.
template <bool BF16>
__device__ __forceinline__ uint32_t instr_desc() {
  uint32_t d = 0;
  d |= 1u << 4;                          // D format f32
  d |= (BF16 ? 1u : 2u) << 7;            // A format: bf16 (kind::f16) or tf32
  d |= (BF16 ? 1u : 2u) << 10;           // B format
  d |= (uint32_t)(BN >> 3) << 17;   // N / 8
  d |= (uint32_t)(BMH >> 4) << 24;  // M / 16 (one half)
  return d;
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

struct TcParams {
  CUtensorMap a_hi[TC_MAXP], a_lo[TC_MAXP], b_hi[TC_MAXP], b_lo[TC_MAXP];
  float* Z[TC_MAXP];
  float* part[TC_MAXP];   // K-split partials of pattern p (splits copies of the Z layout), when splits > 1
  int splits;
  long long ldz[TC_MAXP];
  int n_b[TC_MAXP];
  int n_rhs[TC_MAXP];
  int tiles_m[TC_MAXP];
  int tile_off[TC_MAXP + 1];
  int n_pat;
  int* error;   // device flag: first failing CTA writes its code
};

}  // namespace

// BF16: operands are bf16 pairs (kind::f16, K = 16 per MMA, 32 per 64-byte row), else tf32 pairs
// (kind::tf32, K = 8 per MMA, 16 per row); either way two MMAs of 32 bytes of K cover one row.
template <bool BF16>
__global__ void __launch_bounds__(THREADS, 1) k_tc_gemm(const __grid_constant__ TcParams P) {
  constexpr int BK = ROW_BYTES / (BF16 ? 2 : 4);   // K elements per stage
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* done = empty + STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* n_loaded = abort_flag + 1;     // stages whose TMA loads were issued
  volatile int* n_consumed = abort_flag + 2;   // stages whose full barrier the MMA thread observed

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tile = (int)blockIdx.x / P.splits, sp = (int)blockIdx.x % P.splits;
  int p = 0;
  while (p + 1 < P.n_pat && tile >= P.tile_off[p + 1]) ++p;
  // right-hand-side tiles inner: the CTAs of a wave share few 128-row tiles of S (read from DRAM once, then
  // served from L2 to the other CTAs of the row), and Y (a few tens of MB per pattern) stays in L2
  const int t = tile - P.tile_off[p];
  const int tiles_n = (P.n_rhs[p] + BN - 1) / BN;
  const int m0 = (t / tiles_n) * BM, n0 = (t % tiles_n) * BN;
  const int nk_all = (P.n_b[p] + BK - 1) / BK;
  const int kb0 = (int)((long long)sp * nk_all / P.splits), kb1 = (int)((long long)(sp + 1) * nk_all / P.splits);
  const int nk = kb1 - kb0;   // K steps of this CTA
  const bool two = m0 + BMH < P.n_b[p];   // the second 128-row half has rows of S (else its MMAs are skipped)

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    *n_loaded = 0;
    *n_consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {   // TMEM allocation: two accumulators of BN fp32 columns, by one full warp
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // producer
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      const uint32_t ph = (kb / STAGES) & 1;
      if (kb >= STAGES && !mbar_wait(&empty[s], ph ^ 1)) {
        atomicCAS(P.error, 0, 1);
        *abort_flag = 1;
        break;
      }
      if (*abort_flag) break;
      uint8_t* st = smem + s * STAGE_BYTES;
      mbar_expect_tx(&full[s], STAGE_BYTES);
      const int kx = (kb0 + kb) * BK;
      tma_load_2d(&P.a_hi[p], &full[s], st, kx, m0);
      tma_load_2d(&P.a_lo[p], &full[s], st + TILE_A_BYTES, kx, m0);
      tma_load_2d(&P.b_hi[p], &full[s], st + 2 * TILE_A_BYTES, kx, n0);
      tma_load_2d(&P.b_lo[p], &full[s], st + 2 * TILE_A_BYTES + TILE_B_BYTES, kx, n0);
      *n_loaded = kb + 1;
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    const uint32_t idesc = instr_desc<BF16>();
    int issued = 0;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      const uint32_t ph = (kb / STAGES) & 1;
      if (!mbar_wait(&full[s], ph)) {
        atomicCAS(P.error, 0, 2);
        *abort_flag = 1;
        break;
      }
      *n_consumed = kb + 1;
      if (*abort_flag) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      uint8_t* st = smem + s * STAGE_BYTES;
      const uint64_t bhi = smem_desc(st + 2 * TILE_A_BYTES), blo = smem_desc(st + 2 * TILE_A_BYTES + TILE_B_BYTES);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (h == 1 && !two) break;
        // half h: rows h * 128 .. of the A tiles (8 KB in), accumulator at TMEM column h * BN
        const uint64_t ahi = smem_desc(st + h * (BMH * ROW_BYTES));
        const uint64_t alo = smem_desc(st + TILE_A_BYTES + h * (BMH * ROW_BYTES));
        const uint32_t acc = tmem + (uint32_t)(h * BN);
#pragma unroll
        for (int kk = 0; kk < ROW_BYTES / 32; ++kk) {
          const uint64_t koff = (uint64_t)((kk * 32) >> 4);   // 32 bytes per MMA: 8 tf32 or 16 bf16 of K
          if (BF16) {
            mma_f16(acc, ahi + koff, bhi + koff, idesc, (kb | kk) ? 1u : 0u);
            mma_f16(acc, ahi + koff, blo + koff, idesc, 1u);
            mma_f16(acc, alo + koff, bhi + koff, idesc, 1u);
          } else {
            mma_tf32(acc, ahi + koff, bhi + koff, idesc, (kb | kk) ? 1u : 0u);
            mma_tf32(acc, ahi + koff, blo + koff, idesc, 1u);
            mma_tf32(acc, alo + koff, bhi + koff, idesc, 1u);
          }
        }
      }
      mma_commit(&empty[s]);   // frees the stage once these MMAs have read it
      ++issued;
    }
    mma_commit(done);          // fires when every MMA issued above has completed
  }
  __syncwarp();

  // epilogue: every warp waits for the accumulators, then drains its 32 TMEM lanes of half warp / 4 (a warp
  // reaches the TMEM lanes 32 (warp % 4) .. + 31 only)
  const bool ok = mbar_wait(done, 0);
  if (!ok) atomicCAS(P.error, 0, 3);
  // the TMEM loads below are warp-collective: take the decision for the whole CTA
  const bool drain = __syncthreads_and(ok && !*abort_flag) != 0;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int half = warp >> 2, quad = warp & 3;
  if (drain && (half == 0 || two)) {
    const int row = m0 + half * BMH + quad * 32 + lane;
    // one split: the result; several: this split's partial (added by k_tc_reduce)
    float* Z = P.splits > 1 ? P.part[p] + (size_t)sp * P.n_rhs[p] * P.ldz[p] : P.Z[p];
    const long long ldz = P.ldz[p];
    const int nr = P.n_rhs[p];
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 32) {
      uint32_t v[32];
      const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(half * BN + c0);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
          "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
            "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
            "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < P.n_b[p]) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int c = n0 + c0 + j;
          if (c < nr) Z[(long long)c * ldz + row] = __uint_as_float(v[j]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  // after an abort: wait (bounded) for TMA loads that were issued but never consumed, so no copy is still
  // writing this CTA's shared memory when it exits
  if (threadIdx.x == 0 && *abort_flag) {
    for (int kb = *n_consumed; kb < *n_loaded; ++kb) mbar_wait(&full[kb % STAGES], (kb / STAGES) & 1);
  }
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

// Z = sum of the K-split partials in split order (the first n_b rows of every column), one thread per element
__global__ void k_tc_reduce(const float* __restrict__ part, int splits, long long count, int n_b, long long ld,
                            float* __restrict__ Z) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count || (int)(i % ld) >= n_b) return;
  float acc = part[i];
  for (int q = 1; q < splits; ++q) acc += part[(size_t)q * count + i];
  Z[i] = acc;
}

__global__ void k_split_tf32(const double* __restrict__ x, long long rows, long long cols, long long ld_in,
                             float* __restrict__ hi, float* __restrict__ lo, long long ld_out) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * ld_out) return;
  const long long r = idx / ld_out, c = idx % ld_out;
  float h = 0.f, l = 0.f;
  if (c < cols) {
    const float v = (float)x[r * ld_in + c];
    uint32_t t;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(v));
    h = __uint_as_float(t);
    l = v - h;
  }
  hi[idx] = h;
  lo[idx] = l;
}

// Rows of Y^T = (Lam Pi)^T, split into tf32 pairs: Y^T(i, j) = Lam(j, i) - sum_m E(i, m) A(j, m), with
// Lam(j, i) = X[i * ldx + j] (the transposed storage of the set-up's L_S^{-1}), A = Lam N_b and
// E = N_b (N_b^T N_b)^{-1} (n_b x kd, row-major); columns n_b .. ld_out - 1 are zero.
__global__ void k_pinv_rows_tf32(const double* __restrict__ X, long long ldx, const double* __restrict__ A,
                                 const double* __restrict__ E, int kd, long long nb, float* __restrict__ hi,
                                 float* __restrict__ lo, long long ld_out) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nb * ld_out) return;
  const long long i = idx / ld_out, j = idx % ld_out;
  float h = 0.f, l = 0.f;
  if (j < nb) {
    double v = X[i * ldx + j];
    for (int m = 0; m < kd; ++m) v -= E[i * kd + m] * A[j * kd + m];
    const float f = (float)v;
    uint32_t t;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(f));
    h = __uint_as_float(t);
    l = f - h;
  }
  hi[idx] = h;
  lo[idx] = l;
}

// ------------------------------------------------------------------------------------------------ host
namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static std::mutex mu;
  static EncodeTiledFn fn = nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    FETIRP_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !p) throw Error(5, "cuTensorMapEncodeTiled unavailable");
    fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 2D map over a row-major (rows x cols, leading dimension ld) array of fp32 (esize 4) or bf16 (esize 2); box of
// one 64-byte row of K (16 or 32 elements) x box_rows rows, 64-byte swizzle.
void make_map(CUtensorMap* m, const void* base, long long rows, long long cols, long long ld, int box_rows,
              int esize) {
  if ((reinterpret_cast<uintptr_t>(base) & 15) || (ld * esize) % 16)
    throw Error(1, "tensor-core operand not 16-byte aligned");
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * esize)};
  cuuint32_t box[2] = {(cuuint32_t)(ROW_BYTES / esize), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode_fn()(m, esize == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                           const_cast<void*>(base), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Error(5, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
}

}  // namespace

void split_tf32(const double* x, long long rows, long long cols, long long ld_in, float* hi, float* lo,
                long long ld_out, cudaStream_t s) {
  const long long n = rows * ld_out;
  if (n == 0) return;
  k_split_tf32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, rows, cols, ld_in, hi, lo, ld_out);
  FETIRP_LAUNCH_CHECK();
}
void pinv_rows_tf32(const double* X, long long ldx, const double* A, const double* E, int kd, long long nb,
                    float* hi, float* lo, long long ld_out, cudaStream_t s) {
  const long long n = nb * ld_out;
  if (n == 0) return;
  k_pinv_rows_tf32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(X, ldx, A, E, kd, nb, hi, lo, ld_out);
  FETIRP_LAUNCH_CHECK();
}

void tc_init() {
  static std::mutex mu;
  static bool attr_done[64] = {};
  std::lock_guard<std::mutex> lock(mu);
  int dev = 0;
  FETIRP_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) throw Error(1, "device ordinal out of range");
  if (!attr_done[dev]) {
    FETIRP_CUDA(cudaFuncSetAttribute(k_tc_gemm<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    FETIRP_CUDA(cudaFuncSetAttribute(k_tc_gemm<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    attr_done[dev] = true;
  }
  encode_fn();   // resolve the driver entry point outside any stream capture
}

int tc_ksplits(const TcProblem& T) {
  long long tiles = 0;
  int min_nb = 1 << 30;
  for (int p = 0; p < T.n_pat; ++p)
    if (T.n_rhs[p] > 0 && T.n_b[p] > 0) {
      tiles += (long long)ceil_div(T.n_b[p], BM) * ceil_div(T.n_rhs[p], BN);
      min_nb = std::min(min_nb, T.n_b[p]);
    }
  // two splits fill at most one wave of 152 SMs, and every split keeps >= 16 K steps of 16 elements
  return (tiles > 0 && tiles <= 76 && min_nb >= 2 * 16 * 16) ? 2 : 1;
}

namespace {
void tc_gemm_split(const TcProblem& T, bool bf16, int* d_error, cudaStream_t s) {
  tc_init();
  const int es = bf16 ? 2 : 4;
  // patterns with work only: a structure need not use every pattern of the context (a tensor map of an empty
  // right-hand-side block would be invalid)
  std::vector<int> busy;
  std::vector<long long> zoff(T.n_pat + 1, 0);   // offset of pattern p in the Z layout (the caller's order)
  for (int p = 0; p < T.n_pat; ++p) {
    if (T.n_rhs[p] > 0 && T.n_b[p] > 0) busy.push_back(p);
    zoff[p + 1] = zoff[p] + (long long)T.n_rhs[p] * T.ldy[p];
  }
  int splits = tc_ksplits(T);
  if (splits > 1 && (!T.part || T.part_elems < splits * zoff[T.n_pat])) splits = 1;
  for (int base = 0; base < (int)busy.size(); base += TC_MAXP) {
    TcParams P;
    std::memset(&P, 0, sizeof(P));
    P.n_pat = std::min(TC_MAXP, (int)busy.size() - base);
    P.error = d_error;
    int total = 0;
    for (int i = 0; i < P.n_pat; ++i) {
      const int p = busy[base + i];
      make_map(&P.a_hi[i], T.S_hi[p], T.n_b[p], T.n_b[p], T.lds[p], BM, es);
      make_map(&P.a_lo[i], T.S_lo[p], T.n_b[p], T.n_b[p], T.lds[p], BM, es);
      make_map(&P.b_hi[i], T.Y_hi[p], T.n_rhs[p], T.n_b[p], T.ldy[p], BN, es);
      make_map(&P.b_lo[i], T.Y_lo[p], T.n_rhs[p], T.n_b[p], T.ldy[p], BN, es);
      P.Z[i] = T.Z[p];
      P.part[i] = T.part ? T.part + splits * zoff[p] : nullptr;
      P.ldz[i] = T.ldy[p];
      P.n_b[i] = T.n_b[p];
      P.n_rhs[i] = T.n_rhs[p];
      P.tiles_m[i] = ceil_div(T.n_b[p], BM);
      P.tile_off[i] = total;
      total += P.tiles_m[i] * ceil_div(T.n_rhs[p], BN);
    }
    P.tile_off[P.n_pat] = total;
    P.splits = splits;
    if (total == 0) continue;
    if (bf16) k_tc_gemm<true><<<total * splits, THREADS, SMEM_BYTES, s>>>(P);
    else k_tc_gemm<false><<<total * splits, THREADS, SMEM_BYTES, s>>>(P);
    FETIRP_LAUNCH_CHECK();
    if (splits > 1)
      for (int i = 0; i < P.n_pat; ++i) {
        const long long count = (long long)P.n_rhs[i] * P.ldz[i];
        k_tc_reduce<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(P.part[i], splits, count, P.n_b[i], P.ldz[i],
                                                                    P.Z[i]);
        FETIRP_LAUNCH_CHECK();
      }
  }
}
}  // namespace

void tc_gemm_tf32x3(const TcProblem& T, int* d_error, cudaStream_t s) { tc_gemm_split(T, false, d_error, s); }
void tc_gemm_bf16x3(const TcProblem& T, int* d_error, cudaStream_t s) { tc_gemm_split(T, true, d_error, s); }

// hi = bf16(x) (round to nearest), lo = bf16(x - hi); x is FP64 or FP32, outputs bf16 with leading dimension ld_out
template <typename TI>
__global__ void k_split_bf16(const TI* __restrict__ x, long long rows, long long cols, long long ld_in,
                             __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, long long ld_out) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * ld_out) return;
  const long long r = idx / ld_out, c = idx % ld_out;
  float h = 0.f, l = 0.f;
  if (c < cols) {
    const float v = (float)x[r * ld_in + c];
    h = __bfloat162float(__float2bfloat16_rn(v));
    l = v - h;
  }
  hi[idx] = __float2bfloat16_rn(h);
  lo[idx] = __float2bfloat16_rn(l);
}

template <typename TI>
static void split_bf16_t(const TI* x, long long rows, long long cols, long long ld_in, __nv_bfloat16* hi,
                         __nv_bfloat16* lo, long long ld_out, cudaStream_t s) {
  const long long n = rows * ld_out;
  if (n == 0) return;
  k_split_bf16<TI><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, rows, cols, ld_in, hi, lo, ld_out);
  FETIRP_LAUNCH_CHECK();
}
void split_bf16(const double* x, long long rows, long long cols, long long ld_in, __nv_bfloat16* hi,
                __nv_bfloat16* lo, long long ld_out, cudaStream_t s) {
  split_bf16_t(x, rows, cols, ld_in, hi, lo, ld_out, s);
}
void split_bf16(const float* x, long long rows, long long cols, long long ld_in, __nv_bfloat16* hi,
                __nv_bfloat16* lo, long long ld_out, cudaStream_t s) {
  split_bf16_t(x, rows, cols, ld_in, hi, lo, ld_out, s);
}

}  // namespace fetirp
