// kerdock_internal.cuh -- plan object and device helpers shared by the
// library's translation units (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/kerdock.h"

namespace kd {

constexpr int kMaxLogD = 12;          // d <= 4096
constexpr int kMaxK = 32;             // number of median-of-means batches
constexpr int kRegK = 16;             // batches whose means a finalizer thread holds in registers
constexpr uint32_t kDefaultPollLimit = 1u << 22;  // mbarrier polls before a wait gives up
constexpr int64_t kMaxN = 1 << 24;    // samples per query
// The table buffer starts with a status area: the device status word at byte
// 0 and, from byte kWorkOffset, counters of dynamically scheduled kernels.
constexpr size_t kStatusBytes = 1024;
constexpr size_t kWorkOffset = 256;
constexpr int kWorkCounters = int((kStatusBytes - kWorkOffset) / 4);

// Device status word codes (first error wins).
enum : uint32_t { kStatusOk = 0, kStatusTimeout = 1, kStatusBadIndex = 2 };

// Tunable geometry of the query kernel's row ring (0 = library default).
struct Tuning {
  int ring_kb = 0;  // KiB of shared memory for the row ring
  int crows = 0;    // rows per ring chunk (1, 2, 4 or 8)
};

struct Plan {
  int64_t m = 0, n = 0, d = 0, B = 0, L = 0, ldr = 0;
  int k = 0, dtype = KERDOCK_F32, J = 0, K = 0, S = 0;
  int64_t N = 0;
  int64_t sign_words = 0;  // uint32 words per sign-table row: max(4, d/32)
  int64_t tsign_words = 0;  // words per row of the lane-transposed table: max(32, d/32)
  size_t repr_bytes = 0, table_bytes = 0;
  // bound device memory
  void* repr = nullptr;
  void* table = nullptr;
  cudaStream_t stream = nullptr;
  bool bound = false;
  // preprocess state
  const float* A = nullptr;
  int64_t lda = 0;
  bool preprocessed = false;
  // device properties
  int device = -1;
  int num_sms = 0;
  Tuning tuning;
  uint32_t poll_limit = kDefaultPollLimit;  // query-kernel waits (lowered only by a test hook)

  uint32_t* status() const { return reinterpret_cast<uint32_t*>(table); }
  int* work_counters() const {
    return reinterpret_cast<int*>(static_cast<char*>(table) + kWorkOffset);
  }
  uint32_t* signs() const {
    return reinterpret_cast<uint32_t*>(static_cast<char*>(table) + kStatusBytes);
  }
  // Lane-transposed copy of the sign table for the coefficient step: for basis
  // b, word [g][L] holds in bit t the sign bit of p = 32 (32 g + t) + L.
  uint32_t* tsigns() const { return signs() + (d / 2) * sign_words; }
  size_t elem_bytes() const { return dtype == KERDOCK_BF16 ? 2 : 4; }
};

// Layout of one launch (shared by all its queries): ring geometry and the
// byte offsets of the dynamic shared-memory regions.
struct LaunchCfg {
  int nchunk;            // ring chunks; a chunk holds crows consecutive samples of one query
  int crows;             // rows per chunk (1, 2, 4 or 8)
  int pgroup;            // chunks the producer fills per warp instruction (pgroup * crows <= 32)
  uint32_t slot_bytes;   // ring slot stride: the largest row of the launch
  int64_t xpad;          // floats per x buffer
  int64_t mstride;       // floats per batch-means buffer (K * ldr of the largest query)
  uint32_t off_coef, off_x, off_means, off_mu, off_sel, off_vals, total;
  float* means_gmem;     // per-CTA batch means in global memory when non-null
  uint32_t* status;
  uint32_t poll_limit;   // mbarrier polls before a wait gives up (kDefaultPollLimit)
};

// Everything one query needs, with pointers already offset to that query.
struct QueryDesc {
  const void* R;            // representation of the query's plan
  const uint32_t* tsigns;   // lane-transposed sign table of the plan
  const float* A;           // rows of A for the refinement
  const float* x;           // the query vector (n floats)
  int32_t* out_idx;         // S kept indices
  float* out_val;           // S kept values
  int32_t* out_count;       // one count
  float* mu_out;            // m floats (debug) or null
  int64_t* ells_out;        // N indices (debug) or null
  float* coef_out;          // N coefficients (debug) or null
  int64_t tstride, lda, m, n, d, L, ldr, N, ctr_base;
  uint64_t seed;
  int32_t k, J, K, S, dtype, flags, a_vec4;
  uint32_t row_bytes;
  float eps, inv_J, sqrt_d;
};

// Largest sizes over the queries of one launch.
struct Dims {
  uint32_t row_bytes = 0;  // bytes of one representation row
  int64_t xpad = 32;       // x buffer floats: max(d, 32)
  int64_t ldr = 0;         // representation row stride (elements)
  int64_t S = 0;           // candidate-set size
  int64_t KL = 0;          // K * ldr
  int coef_warps = 3;      // coefficient warps of the kernel that runs (3: batch kernel)
};

size_t align_up(size_t v, size_t al);
void dims_add(Dims& dm, const Plan& p, int64_t K, int64_t S);
Dims plan_dims(const Plan& p);  // one plan's dims with its single-plan kernel's split
bool means_fit_smem(const Dims& dm);
// packed: the batch kernel, whose chunks may pack several small rows per slot
bool make_cfg(const Dims& dm, const Tuning& tu, bool means_in_smem, LaunchCfg& c,
              bool packed = false);
QueryDesc plan_desc(const Plan& p);
void set_query_params(QueryDesc& d, int64_t J, int64_t K, int64_t S, float eps, uint64_t seed,
                      int flags);
int prepare_batch_kernel(const LaunchCfg& cfg);  // kernel attributes; call outside capture
int launch_batch(const LaunchCfg& cfg, const QueryDesc* descs, const int32_t* order,
                 const int64_t* cta_start, int grid, cudaStream_t stream);
constexpr int kQueryThreads = 512;

// C[M x N] (float32, row stride ldc) = sum_k A(m, k) B(n, k) on the tensor
// cores (bfloat16 operands, float32 accumulation; mlp.cu).
struct GemmArgs {
  int M, N, K;
  const __nv_bfloat16* A;  // element (m, k) at A[m * sAm + k * sAk]
  int64_t sAm, sAk;
  const __nv_bfloat16* B;  // element (n, k) at B[n * sBn + k * sBk]
  int64_t sBn, sBk;
  int kc;  // k range of one slice when K is split (a multiple of 64), 0: no split
  uint32_t* status = nullptr;  // device status word for a bounded wait that ran out
};

// Split of K into slices so that a small M x N product still puts about two
// 128 x 64 tiles on every SM: slice z covers k in [z kc, (z + 1) kc) and writes
// its partial product to its own M x N plane; the reader sums the planes in
// order z = 0, 1, ... (deterministic).
struct GemmSplit {
  int slices, kc;
};
GemmSplit gemm_split(int64_t M, int64_t N, int64_t K, int num_sms);
// The split product: plane z at C + z * plane (row stride ldc).
int gemm_bf16_f32_split(GemmArgs g, const GemmSplit& sp, float* C, int64_t ldc, int64_t plane,
                        cudaStream_t stream);

// Launchers (return KERDOCK_OK or a negative error code).
int launch_signs(const Plan& p);
int launch_preprocess(const Plan& p);
int launch_apply(const Plan& p, const float* X, int64_t q, int64_t ldx, float eps,
                 uint64_t seed, int flags, int32_t* out_idx, float* out_val,
                 int32_t* out_count, void* ws, size_t ws_bytes, float* mu_out,
                 int64_t* ells_out, float* coef_out);
size_t apply_workspace_bytes(const Plan& p, int64_t q);
int launch_apply_noalloc(const Plan& p, const float* X, int64_t q, int64_t ldx, float eps,
                         uint64_t seed, int flags, int32_t* out_idx, float* out_val,
                         int32_t* out_count);
size_t noalloc_scratch_bytes();

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------

// Record the first device-side error in the plan's status word.
__device__ __forceinline__ void set_status(uint32_t* status, uint32_t code) {
  atomicCAS(status, kStatusOk, code);
}

// SplitMix64 output function (Steele, Lea & Flood, OOPSLA 2014).
__device__ __forceinline__ uint64_t splitmix64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Sample index l_j of the counter-based sampling convention of kerdock.h.
__device__ __forceinline__ uint64_t sample_index(uint64_t seed, uint64_t ctr, uint64_t L) {
  const uint64_t z = splitmix64_mix(seed + 0x9E3779B97F4A7C15ull * (ctr + 1));
  return __umul64hi(z, L);
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count));
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

// Raise the phase's expected transaction bytes without arriving.
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase.  Returns false after ~2^22 polls (each
// try_wait itself blocks for a hardware-defined slice), i.e. seconds.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  for (uint32_t it = 0; it < (1u << 22); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
  }
  return false;
}

// Bulk prefetch of a contiguous global range into L2 (TMA engine, no
// registers, no completion).  src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// 1-D bulk copy global -> shared (TMA engine), completion on an mbarrier.
// dst/src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float flip_sign(float v, uint32_t bit) {
  return __uint_as_float(__float_as_uint(v) ^ (bit << 31));
}

}  // namespace kd

struct kerdock_plan_s {
  kd::Plan p;
};

#define KD_CUDA_TRY(expr)                           \
  do {                                              \
    cudaError_t kd_err_ = (expr);                   \
    if (kd_err_ != cudaSuccess) return KERDOCK_ERR_CUDA; \
  } while (0)
