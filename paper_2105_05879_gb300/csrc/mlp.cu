// mlp.cu -- the learned-proposal network and the bfloat16 tensor-core GEMMs.
//
// Not in the paper: a project form that replaces the |mu| ranking of
// Algorithm 1's top-S step by the scores of a small network fed with a cheap
// sketch mu (reduced N), so that fewer samples and fewer refined rows reach the
// same support.  The network is a three-layer perceptron in bfloat16 with FP32
// accumulation on the tensor cores, trained on the GPU with
// binary cross-entropy on logits and AdamW:
//   H1 = relu(X W1^T + b1), H2 = relu(H1 W2^T + b2), Z = H2 W3^T + b3.
// Every product of the forward and backward passes is one strided GEMM
// C = op(A) op(B)^T with a fused epilogue (bias, ReLU, ReLU mask, FP32/BF16).
// Products of two k-major operands (the forward layers, the shared-sample
// query's products) run on tcgen05 with TMA-fed operands and a tensor-memory
// accumulator; the transposed operands of the backward pass take a cp.async +
// ldmatrix + mma.sync kernel.
#include <cuda.h>  // CUtensorMap (types only; the encoder comes from the runtime)

#include <algorithm>
#include <cstring>
#include <new>

#include "kerdock_internal.cuh"

namespace kd {
namespace {

constexpr int GBM = 64, GBN = 64, GBK = 32, GTHREADS = 128;

__device__ __forceinline__ uint32_t ld_pair(const __nv_bfloat16* p) {
  return *reinterpret_cast<const uint32_t*>(p);
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// C[m, n] = sum_k A(m, k) B(n, k), 64 x 64 tiles, 4 warps of 32 x 32, epilogue
// functor per element.
template <class Epi>
__global__ void __launch_bounds__(GTHREADS) gemm_bf16_kernel(const GemmArgs g, const Epi epi) {
  __shared__ __align__(16) __nv_bfloat16 As[GBM][GBK + 8];
  __shared__ __align__(16) __nv_bfloat16 Bs[GBN][GBK + 8];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int group = lane >> 2, tig = lane & 3;
  const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
  const int wm = (warp & 1) * 32, wn = (warp >> 1) * 32;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
  const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
  const int kbeg = g.kc ? int(blockIdx.z) * g.kc : 0;
  const int kend = g.kc ? min(g.K, kbeg + g.kc) : g.K;
  for (int k0 = kbeg; k0 < kend; k0 += GBK) {
    for (int i = tid; i < GBM * GBK; i += GTHREADS) {
      int mm, kk;
      if (g.sAk == 1) { mm = i / GBK; kk = i % GBK; } else { mm = i % GBM; kk = i / GBM; }
      const int gm = m0 + mm, gk = k0 + kk;
      As[mm][kk] = (gm < g.M && gk < kend) ? g.A[int64_t(gm) * g.sAm + int64_t(gk) * g.sAk] : zero;
    }
    for (int i = tid; i < GBN * GBK; i += GTHREADS) {
      int nn, kk;
      if (g.sBk == 1) { nn = i / GBK; kk = i % GBK; } else { nn = i % GBN; kk = i / GBN; }
      const int gn = n0 + nn, gk = k0 + kk;
      Bs[nn][kk] = (gn < g.N && gk < kend) ? g.B[int64_t(gn) * g.sBn + int64_t(gk) * g.sBk] : zero;
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < GBK; ks += 16) {
      uint32_t a[2][4], b[4][2];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const int r = wm + mt * 16 + group, c = ks + tig * 2;
        a[mt][0] = ld_pair(&As[r][c]);
        a[mt][1] = ld_pair(&As[r + 8][c]);
        a[mt][2] = ld_pair(&As[r][c + 8]);
        a[mt][3] = ld_pair(&As[r + 8][c + 8]);
      }
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int r = wn + nt * 8 + group, c = ks + tig * 2;
        b[nt][0] = ld_pair(&Bs[r][c]);
        b[nt][1] = ld_pair(&Bs[r][c + 8]);
      }
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
          mma_bf16(acc[mt][nt], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b[nt][0], b[nt][1]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = m0 + wm + mt * 16 + group + (e >= 2 ? 8 : 0);
        const int c = n0 + wn + nt * 8 + tig * 2 + (e & 1);
        if (r < g.M && c < g.N) epi(r, c, acc[mt][nt][e]);
      }
}

// The same product for 16-byte-aligned operands: each operand tile is moved by
// cp.async in 16-byte pieces along its contiguous dimension (k for a
// "k-major" operand, m or n otherwise) through a GSTAGES-deep shared-memory
// ring, and the mma fragments are read with ldmatrix (.trans for the
// m/n-major tiles).  Pieces past the matrix edge are zero-filled by the copy
// itself (source size below 16 bytes), so ragged M, N and K need no branch in
// the inner loop.
constexpr int GSTAGES = 4;
constexpr int KM_LD = GBK + 8;   // k-major tile [rows][GBK], padded: 80-byte rows
constexpr int MM_LD = GBM + 8;   // m/n-major tile [GBK][rows], padded: 144-byte rows
constexpr int TILE_ELEMS = GBM * KM_LD > GBK * MM_LD ? GBM * KM_LD : GBK * MM_LD;
static_assert(GBM == GBN, "one tile shape serves both operands");

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t (&r)[4]) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t (&r)[4]) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}

// Issue the copies of one GBK slice of a GBM-row operand tile: rows r0.., k0..
// of a rows x K matrix with element (r, k) at P[r * s_r + k * s_k].
template <bool KMAJOR>
__device__ __forceinline__ void load_tile(__nv_bfloat16* dst, const __nv_bfloat16* P, int64_t s_r,
                                          int64_t s_k, int rows, int K, int r0, int k0, int tid) {
  constexpr int PIECES = GBM * GBK / 8;
#pragma unroll
  for (int c = tid; c < PIECES; c += GTHREADS) {
    int rr, kk, bytes;
    const __nv_bfloat16* src = P;
    uint32_t d;
    if (KMAJOR) {  // piece = 8 consecutive k of one row
      rr = c / (GBK / 8);
      kk = (c % (GBK / 8)) * 8;
      const int gr = r0 + rr, gk = k0 + kk;
      bytes = (gr < rows && gk < K) ? 2 * min(8, K - gk) : 0;
      if (bytes) src = P + int64_t(gr) * s_r + gk;
      d = smem_addr(dst + rr * KM_LD + kk);
    } else {  // piece = 8 consecutive rows of one k
      kk = c / (GBM / 8);
      rr = (c % (GBM / 8)) * 8;
      const int gr = r0 + rr, gk = k0 + kk;
      bytes = (gk < K && gr < rows) ? 2 * min(8, rows - gr) : 0;
      if (bytes) src = P + int64_t(gk) * s_k + gr;
      d = smem_addr(dst + kk * MM_LD + rr);
    }
    cp_async16(d, src, bytes);
  }
}

template <bool AK, bool BK, class Epi>
__global__ void __launch_bounds__(GTHREADS) gemm_bf16_async_kernel(const GemmArgs g,
                                                                   const Epi epi) {
  __shared__ __align__(128) __nv_bfloat16 As[GSTAGES][TILE_ELEMS];
  __shared__ __align__(128) __nv_bfloat16 Bs[GSTAGES][TILE_ELEMS];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int group = lane >> 2, tig = lane & 3;
  const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
  const int wm = (warp & 1) * 32, wn = (warp >> 1) * 32;
  const int kbeg = g.kc ? int(blockIdx.z) * g.kc : 0;
  const int kend = g.kc ? min(g.K, kbeg + g.kc) : g.K;
  const int ktiles = (kend - kbeg + GBK - 1) / GBK;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
  auto issue = [&](int kt) {
    if (kt < ktiles) {
      const int s = kt % GSTAGES;
      load_tile<AK>(As[s], g.A, g.sAm, g.sAk, g.M, kend, m0, kbeg + kt * GBK, tid);
      load_tile<BK>(Bs[s], g.B, g.sBn, g.sBk, g.N, kend, n0, kbeg + kt * GBK, tid);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
#pragma unroll
  for (int s = 0; s < GSTAGES - 1; ++s) issue(s);
  const int j8 = lane >> 3, r8 = lane & 7;
  for (int kt = 0; kt < ktiles; ++kt) {
    asm volatile("cp.async.wait_group %0;" ::"n"(GSTAGES - 2) : "memory");
    __syncthreads();  // slice kt visible to all; slot of kt - 1 free again
    issue(kt + GSTAGES - 1);
    const __nv_bfloat16* a_s = As[kt % GSTAGES];
    const __nv_bfloat16* b_s = Bs[kt % GSTAGES];
#pragma unroll
    for (int ks = 0; ks < GBK; ks += 16) {
      uint32_t a[2][4], b[4][2];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        // matrices in fragment order: (m 0-7, k 0-7), (m 8-15, k 0-7),
        // (m 0-7, k 8-15), (m 8-15, k 8-15)
        if (AK)
          ldsm_x4(smem_addr(a_s + (wm + mt * 16 + (lane & 15)) * KM_LD + ks + (lane >> 4) * 8),
                  a[mt]);
        else
          ldsm_x4_t(smem_addr(a_s + (ks + (j8 >> 1) * 8 + r8) * MM_LD + wm + mt * 16 +
                              (j8 & 1) * 8),
                    a[mt]);
      }
#pragma unroll
      for (int np = 0; np < 2; ++np) {
        // matrices: (n 0-7, k 0-7), (n 0-7, k 8-15), (n 8-15, k 0-7), (n 8-15, k 8-15)
        uint32_t t[4];
        const int nb = wn + np * 16 + (j8 >> 1) * 8, kb = ks + (j8 & 1) * 8;
        if (BK)
          ldsm_x4(smem_addr(b_s + (nb + r8) * KM_LD + kb), t);
        else
          ldsm_x4_t(smem_addr(b_s + (kb + r8) * MM_LD + nb), t);
        b[2 * np][0] = t[0];
        b[2 * np][1] = t[1];
        b[2 * np + 1][0] = t[2];
        b[2 * np + 1][1] = t[3];
      }
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
          mma_bf16(acc[mt][nt], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b[nt][0], b[nt][1]);
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = m0 + wm + mt * 16 + group + (e >= 2 ? 8 : 0);
        const int c = n0 + wn + nt * 8 + tig * 2 + (e & 1);
        if (r < g.M && c < g.N) epi(r, c, acc[mt][nt][e]);
      }
}

// ---------------------------------------------------------------------------
// The same product on the fifth-generation tensor cores for two k-major
// operands (both 16-byte aligned with 16-byte row pitches): a 128 x 64 output
// tile per CTA, accumulated in 64 columns of tensor memory by tcgen05.mma
// (kind::f16, bfloat16 in, float32 out).  One thread streams 128 x 64 and
// 64 x 64 operand blocks into a TC_STAGES-deep shared-memory ring with TMA
// (128-byte swizzle, zero fill past the matrix edges), one thread issues the
// MMAs (four K = 16 steps per block) and returns each slot with
// tcgen05.commit, and the four warps read the accumulator back (warp w owns
// tensor-memory lanes 32w .. 32w + 31 = tile rows) for the epilogue.  Every
// wait is bounded; a wait that runs out records a timeout in the status word
// (when the caller gives one) and the CTA drains its issued work before it
// frees the tensor memory.
constexpr int TC_M = 128, TC_N = 64, TC_K = 64, TC_STAGES = 4, TC_THREADS = 128;
constexpr uint32_t TC_A_BYTES = TC_M * TC_K * 2, TC_B_BYTES = TC_N * TC_K * 2;
constexpr uint32_t TC_STAGE_BYTES = TC_A_BYTES + TC_B_BYTES;
constexpr uint32_t TC_SMEM = 1024 + TC_STAGES * TC_STAGE_BYTES + 256;
constexpr uint32_t TC_TMEM_COLS = 64;
// instruction descriptor (kind::f16): D float32, A and B bfloat16, both
// k-major, N >> 3 at bit 17, M >> 4 at bit 24
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(TC_N >> 3) << 17) |
                              (uint32_t(TC_M >> 4) << 24);

// Shared-memory matrix descriptor of a k-major operand block in the 128-byte
// swizzled layout that TMA writes: rows of 128 bytes, 8-row groups 1024 bytes
// apart (stride byte offset), block base 1024-byte aligned.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  return uint64_t((saddr >> 4) & 0x3FFFu) | (uint64_t(1) << 16) | (uint64_t(1024 >> 4) << 32) |
         (uint64_t(1) << 46) | (uint64_t(2) << 61);
}

__device__ __forceinline__ void tc_tma_load(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, "
      "{%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(TC_IDESC), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]),
                 "+r"(v[6]), "+r"(v[7]), "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]),
                 "+r"(v[12]), "+r"(v[13]), "+r"(v[14]), "+r"(v[15])
               :
               : "memory");
}

template <class Epi>
__global__ void __launch_bounds__(TC_THREADS)
    gemm_tc_kernel(const GemmArgs g, const Epi epi, const __grid_constant__ CUtensorMap tmA,
                   const __grid_constant__ CUtensorMap tmB) {
  extern __shared__ unsigned char tc_smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + TC_STAGES * TC_STAGE_BYTES);
  uint64_t* empty = full + TC_STAGES;
  uint64_t* done = empty + TC_STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m0 = blockIdx.y * TC_M, n0 = blockIdx.x * TC_N;
  const int kbeg = g.kc ? int(blockIdx.z) * g.kc : 0;
  const int kend = g.kc ? min(g.K, kbeg + g.kc) : g.K;
  const int ktiles = (kend - kbeg + TC_K - 1) / TC_K;
  const uint32_t sbase = smem_addr(sm);

  if (tid == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(tmem_slot)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(tmem_slot);

  bool ok = true;
  if (tid == 0) {  // TMA producer
    int issued = 0;
    for (int kt = 0; kt < ktiles; ++kt) {
      const int s = kt % TC_STAGES;
      if (kt >= TC_STAGES && !mbar_wait_bounded(&empty[s], uint32_t((kt / TC_STAGES) - 1) & 1u)) {
        ok = false;
        break;
      }
      mbar_arrive_expect_tx(&full[s], TC_STAGE_BYTES);
      const uint32_t a_s = sbase + s * TC_STAGE_BYTES;
      tc_tma_load(a_s, &tmA, kbeg + kt * TC_K, m0, &full[s]);
      tc_tma_load(a_s + TC_A_BYTES, &tmB, kbeg + kt * TC_K, n0, &full[s]);
      issued = kt + 1;
    }
    // the copies still in flight land before the CTA can leave
    for (int kt = issued - TC_STAGES > 0 ? issued - TC_STAGES : 0; kt < issued; ++kt)
      if (!mbar_wait_bounded(&full[kt % TC_STAGES], uint32_t(kt / TC_STAGES) & 1u)) ok = false;
  } else if (tid == 32) {  // MMA issuer
    for (int kt = 0; kt < ktiles; ++kt) {
      const int s = kt % TC_STAGES;
      if (!mbar_wait_bounded(&full[s], uint32_t(kt / TC_STAGES) & 1u)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a_s = sbase + s * TC_STAGE_BYTES;
      const uint64_t ad = tc_desc(a_s), bd = tc_desc(a_s + TC_A_BYTES);
#pragma unroll
      for (int kk = 0; kk < TC_K / 16; ++kk)  // +32 bytes per K = 16 step inside the swizzle row
        tc_mma(tmem, ad + uint64_t(kk * 2), bd + uint64_t(kk * 2), (kt | kk) != 0 ? 1u : 0u);
      tc_commit(&empty[s]);
    }
    tc_commit(done);  // fires when every MMA issued above has completed
  }
  __syncwarp();
  const bool have = mbar_wait_bounded(done, 0);
  __syncwarp();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (have) {
    // the ring is idle once every MMA has completed: each warp parks its 32
    // accumulator rows there (row pitch 65 words, no bank conflicts) and
    // writes them back row by row, 32 consecutive columns per instruction
    float* park = reinterpret_cast<float*>(sm) + warp * 32 * (TC_N + 1);
    const uint32_t trow = tmem + (uint32_t(warp * 32) << 16);
#pragma unroll
    for (int c0 = 0; c0 < TC_N; c0 += 16) {
      uint32_t v[16];
      tc_ld16(trow + uint32_t(c0), v);
#pragma unroll
      for (int j = 0; j < 16; ++j)
        park[lane * (TC_N + 1) + c0 + j] = ktiles > 0 ? __uint_as_float(v[j]) : 0.f;
    }
    __syncwarp();
    for (int rr = 0; rr < 32; ++rr) {
      const int r = m0 + warp * 32 + rr;
      if (r >= g.M) break;
#pragma unroll
      for (int c = lane; c < TC_N; c += 32)
        if (n0 + c < g.N) epi(r, n0 + c, park[rr * (TC_N + 1) + c]);
    }
  }
  if ((!ok || !have) && g.status != nullptr) set_status(g.status, kStatusTimeout);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TC_TMEM_COLS)
                 : "memory");
}

struct EpiBiasReluBf16 {  // C = bf16(relu(acc + bias[c]))
  const float* bias;
  __nv_bfloat16* C;
  int ldc;
  __device__ void operator()(int r, int c, float v) const {
    v += bias[c];
    C[int64_t(r) * ldc + c] = __float2bfloat16_rn(v > 0.f ? v : 0.f);
  }
};
struct EpiBiasF32 {  // C = acc + bias[c] (+ skip * X[r, c] when skip != 0: residual logits)
  const float* bias;
  float* C;
  int ldc;
  const __nv_bfloat16* X;
  float skip;
  __device__ void operator()(int r, int c, float v) const {
    const int64_t i = int64_t(r) * ldc + c;
    C[i] = v + bias[c] + (skip != 0.f ? skip * __bfloat162float(X[i]) : 0.f);
  }
};
struct EpiMaskBf16 {  // C = bf16(acc) where H > 0, else 0 (ReLU derivative, relu'(0) = 0)
  const __nv_bfloat16* H;
  __nv_bfloat16* C;
  int ld;
  __device__ void operator()(int r, int c, float v) const {
    const int64_t i = int64_t(r) * ld + c;
    C[i] = __bfloat162float(H[i]) > 0.f ? __float2bfloat16_rn(v) : __float2bfloat16_rn(0.f);
  }
};
struct EpiF32 {  // C = acc (slice z of a split product into plane z)
  float* C;
  int64_t ldc, plane;
  __device__ void operator()(int r, int c, float v) const {
    C[int64_t(blockIdx.z) * plane + int64_t(r) * ldc + c] = v;
  }
};

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn tensor_map_encoder() {
  static EncodeTiledFn fn = nullptr;
  if (fn == nullptr) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult qr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &qr) == cudaSuccess &&
        qr == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(f);
  }
  return fn;
}

// rows x K bfloat16 k-major operand (row pitch `pitch` elements) as a 2-D
// tensor map with a K_block x rows_block box in the 128-byte swizzle
bool encode_kmajor(CUtensorMap* map, const __nv_bfloat16* base, int rows, int K, int64_t pitch,
                   uint32_t box_rows) {
  EncodeTiledFn enc = tensor_map_encoder();
  if (enc == nullptr) return false;
  const cuuint64_t dims[2] = {cuuint64_t(K), cuuint64_t(rows)};
  const cuuint64_t strides[1] = {cuuint64_t(pitch) * 2};
  const cuuint32_t box[2] = {uint32_t(TC_K), box_rows};
  const cuuint32_t es[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(base), dims,
             strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The tcgen05 kernel when both operands are k-major with 16-byte rows;
// `used` is false when the tensor maps cannot be made (the caller falls back).
template <class Epi>
int gemm_tc(const GemmArgs& g, const Epi& epi, cudaStream_t stream, bool& used) {
  used = false;
  CUtensorMap ma, mb;
  if (!encode_kmajor(&ma, g.A, g.M, g.K, g.sAm, TC_M) ||
      !encode_kmajor(&mb, g.B, g.N, g.K, g.sBn, TC_N))
    return KERDOCK_OK;
  static int attr_device = -1;  // one per epilogue type, set on the device in use
  int device = 0;
  KD_CUDA_TRY(cudaGetDevice(&device));
  if (attr_device != device) {
    KD_CUDA_TRY(cudaFuncSetAttribute(gemm_tc_kernel<Epi>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, int(TC_SMEM)));
    attr_device = device;
  }
  const unsigned slices = g.kc ? unsigned((g.K + g.kc - 1) / g.kc) : 1u;
  const dim3 grid(unsigned((g.N + TC_N - 1) / TC_N), unsigned((g.M + TC_M - 1) / TC_M), slices);
  gemm_tc_kernel<Epi><<<grid, TC_THREADS, TC_SMEM, stream>>>(g, epi, ma, mb);
  KD_CUDA_TRY(cudaGetLastError());
  used = true;
  return KERDOCK_OK;
}

// Two k-major operands with 16-byte rows take the tcgen05 kernel; other
// operands whose rows along the contiguous dimension start on 16-byte
// boundaries the cp.async kernel; any other layout the element-wise one.
template <class Epi>
int gemm(const GemmArgs& g, const Epi& epi, cudaStream_t stream) {
  const unsigned slices = g.kc ? unsigned((g.K + g.kc - 1) / g.kc) : 1u;
  const dim3 grid(unsigned((g.N + GBN - 1) / GBN), unsigned((g.M + GBM - 1) / GBM), slices);
  auto aligned16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
  const bool ak = g.sAk == 1 && g.sAm % 8 == 0, am = g.sAm == 1 && g.sAk % 8 == 0;
  const bool bk = g.sBk == 1 && g.sBn % 8 == 0, bn = g.sBn == 1 && g.sBk % 8 == 0;
  if (ak && bk && aligned16(g.A) && aligned16(g.B)) {
    bool used = false;
    const int rc = gemm_tc(g, epi, stream, used);
    if (rc != KERDOCK_OK || used) return rc;
  }
  if ((ak || am) && (bk || bn) && aligned16(g.A) && aligned16(g.B)) {
    if (ak && bk)
      gemm_bf16_async_kernel<true, true, Epi><<<grid, GTHREADS, 0, stream>>>(g, epi);
    else if (ak)
      gemm_bf16_async_kernel<true, false, Epi><<<grid, GTHREADS, 0, stream>>>(g, epi);
    else if (bk)
      gemm_bf16_async_kernel<false, true, Epi><<<grid, GTHREADS, 0, stream>>>(g, epi);
    else
      gemm_bf16_async_kernel<false, false, Epi><<<grid, GTHREADS, 0, stream>>>(g, epi);
  } else {
    gemm_bf16_kernel<Epi><<<grid, GTHREADS, 0, stream>>>(g, epi);
  }
  KD_CUDA_TRY(cudaGetLastError());
  return KERDOCK_OK;
}

// features = bf16(scale * mu), or bf16(scale * |mu|) in magnitude mode
__global__ void to_bf16_kernel(const float* __restrict__ x, int64_t count, float scale, int abs_mode,
                               __nv_bfloat16* __restrict__ y) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < count;
       i += int64_t(gridDim.x) * blockDim.x)
    y[i] = __float2bfloat16_rn(scale * (abs_mode ? fabsf(x[i]) : x[i]));
}

// BCE with logits: dZ = (w+ y (sigmoid(z) - 1) + (1 - y) sigmoid(z)) / B, and the
// summed loss (w+ y softplus(-z) + (1 - y) softplus(z)) / B into *loss.
__global__ void bce_kernel(const float* __restrict__ Z, const float* __restrict__ Y,
                           int64_t count, float inv_B, float pos_weight,
                           __nv_bfloat16* __restrict__ dZ, float* __restrict__ loss) {
  float part = 0.f;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < count;
       i += int64_t(gridDim.x) * blockDim.x) {
    const float z = Z[i], y = Y[i];
    const float sig = 1.f / (1.f + expf(-z));
    dZ[i] = __float2bfloat16_rn((pos_weight * y * (sig - 1.f) + (1.f - y) * sig) * inv_B);
    const float sp_pos = fmaxf(z, 0.f) + log1pf(expf(-fabsf(z)));  // softplus(z)
    const float sp_neg = sp_pos - z;                                // softplus(-z)
    part += (pos_weight * y * sp_neg + (1.f - y) * sp_pos) * inv_B;
  }
  part = warp_sum(part);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, part);
}

// db[n] = sum_b dY[b, n]
__global__ void bias_grad_kernel(const __nv_bfloat16* __restrict__ dY, int B, int N,
                                 float* __restrict__ db) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int b = 0; b < B; ++b) s += __bfloat162float(dY[int64_t(b) * N + n]);
  db[n] = s;
}

// AdamW over all parameters (decoupled weight decay); refreshes the bf16 copy
// of the weight matrices.
struct AdamArgs {
  float* p;
  const float* g;
  float* m;
  float* v;
  int64_t count;
  float lr, beta1, beta2, eps, wd, c1, c2;  // c1 = 1/(1-beta1^t), c2 = 1/(1-beta2^t)
  int64_t w_begin[3], w_end[3];             // weight-matrix ranges in p
  __nv_bfloat16* wbf[3];                    // their bf16 copies
};

__global__ void adamw_kernel(const AdamArgs a) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < a.count;
       i += int64_t(gridDim.x) * blockDim.x) {
    const float g = a.g[i];
    const float m = a.beta1 * a.m[i] + (1.f - a.beta1) * g;
    const float v = a.beta2 * a.v[i] + (1.f - a.beta2) * g * g;
    a.m[i] = m;
    a.v[i] = v;
    const float p = a.p[i] - a.lr * ((m * a.c1) / (sqrtf(v * a.c2) + a.eps) + a.wd * a.p[i]);
    a.p[i] = p;
#pragma unroll
    for (int w = 0; w < 3; ++w)
      if (i >= a.w_begin[w] && i < a.w_end[w]) a.wbf[w][i - a.w_begin[w]] = __float2bfloat16_rn(p);
  }
}

// Uniform(-bound, bound) initial weights from the SplitMix64 counter hash, zero
// biases and optimiser moments.
__global__ void init_kernel(float* __restrict__ p, int64_t count, uint64_t seed,
                            const int64_t* __restrict__ seg_end, const float* __restrict__ bound,
                            int nseg) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < count;
       i += int64_t(gridDim.x) * blockDim.x) {
    int s = 0;
    while (s < nseg - 1 && i >= seg_end[s]) ++s;
    const uint64_t z = splitmix64_mix(seed + 0x9E3779B97F4A7C15ull * uint64_t(i + 1));
    const float u = float(z >> 40) * (1.0f / 16777216.0f);  // [0, 1)
    p[i] = bound[s] * (2.f * u - 1.f);
  }
}

__global__ void f32_to_bf16_kernel(const float* __restrict__ x, int64_t count,
                                   __nv_bfloat16* __restrict__ y) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < count;
       i += int64_t(gridDim.x) * blockDim.x)
    y[i] = __float2bfloat16_rn(x[i]);
}

unsigned grid_for(int64_t count, int threads) {
  int64_t g = (count + threads - 1) / threads;
  if (g > 4096) g = 4096;
  return unsigned(g < 1 ? 1 : g);
}

}  // namespace

GemmSplit gemm_split(int64_t M, int64_t N, int64_t K, int num_sms) {
  // sized for the tcgen05 tiles (128 x 64, k blocks of 64; two CTAs per SM)
  const int64_t tiles = ((M + TC_M - 1) / TC_M) * ((N + TC_N - 1) / TC_N);
  const int64_t kblocks = (K + TC_K - 1) / TC_K;
  int64_t s = (2 * int64_t(num_sms) + tiles - 1) / tiles;
  s = std::min<int64_t>(s, std::max<int64_t>(1, kblocks / 4));  // >= 4 k blocks per slice
  s = std::max<int64_t>(1, std::min<int64_t>(s, 8));
  GemmSplit sp;
  sp.kc = int((kblocks + s - 1) / s) * TC_K;
  sp.slices = int((K + sp.kc - 1) / sp.kc);
  return sp;
}

int gemm_bf16_f32_split(GemmArgs g, const GemmSplit& sp, float* C, int64_t ldc, int64_t plane,
                        cudaStream_t stream) {
  if (g.M < 1 || g.N < 1 || g.K < 1) return KERDOCK_OK;
  g.kc = sp.slices > 1 ? sp.kc : 0;
  return gemm(g, EpiF32{C, ldc, plane}, stream);
}

}  // namespace kd

struct kerdock_mlp_s {
  int in = 0, hid = 0, out = 0, max_batch = 0;
  int64_t off[7] = {};  // parameter offsets: W1, b1, W2, b2, W3, b3, end
  int64_t count = 0;    // parameters
  size_t state_bytes = 0, work_bytes = 0;
  // state
  float* master = nullptr;
  float* grads = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  __nv_bfloat16* wbf[3] = {};
  float* loss = nullptr;
  // work
  __nv_bfloat16* X0 = nullptr;
  __nv_bfloat16* H1 = nullptr;
  __nv_bfloat16* H2 = nullptr;
  float* Z = nullptr;
  __nv_bfloat16* dZ = nullptr;
  __nv_bfloat16* dH2 = nullptr;
  __nv_bfloat16* dH1 = nullptr;
  cudaStream_t stream = nullptr;
  bool bound = false;
  int64_t step = 0;
  int input_mode = 0;  // KERDOCK_MLP_INPUT_*
  float skip = 0.f;    // residual logits Z += skip * X (needs in_dim == out_dim)
};

namespace {

size_t a256(size_t v) { return (v + 255) / 256 * 256; }

int mlp_forward_impl(kerdock_mlp_s* n, const float* feats, int B, float scale, float* logits) {
  using namespace kd;
  to_bf16_kernel<<<grid_for(int64_t(B) * n->in, 256), 256, 0, n->stream>>>(
      feats, int64_t(B) * n->in, scale, n->input_mode == KERDOCK_MLP_INPUT_ABS, n->X0);
  KD_CUDA_TRY(cudaGetLastError());
  GemmArgs g{};
  // H1 = relu(X0 W1^T + b1)
  g = GemmArgs{B, n->hid, n->in, n->X0, n->in, 1, n->wbf[0], n->in, 1};
  int rc = gemm(g, EpiBiasReluBf16{n->master + n->off[1], n->H1, n->hid}, n->stream);
  if (rc != KERDOCK_OK) return rc;
  // H2 = relu(H1 W2^T + b2)
  g = GemmArgs{B, n->hid, n->hid, n->H1, n->hid, 1, n->wbf[1], n->hid, 1};
  rc = gemm(g, EpiBiasReluBf16{n->master + n->off[3], n->H2, n->hid}, n->stream);
  if (rc != KERDOCK_OK) return rc;
  // Z = H2 W3^T + b3
  g = GemmArgs{B, n->out, n->hid, n->H2, n->hid, 1, n->wbf[2], n->hid, 1};
  return gemm(g, EpiBiasF32{n->master + n->off[5], logits, n->out, n->X0, n->skip}, n->stream);
}

}  // namespace

extern "C" {

int kerdock_mlp_create(kerdock_mlp_t* mlp, int32_t in_dim, int32_t hidden, int32_t out_dim,
                       int32_t max_batch) {
  if (mlp == nullptr) return KERDOCK_ERR_INVALID_ARG;
  *mlp = nullptr;
  if (in_dim < 1 || hidden < 1 || out_dim < 1 || max_batch < 1) return KERDOCK_ERR_INVALID_ARG;
  if (in_dim % 2 || hidden % 2 || out_dim % 2 || in_dim > 65536 || hidden > 65536 ||
      out_dim > 65536 || max_batch > 1 << 20)
    return KERDOCK_ERR_UNSUPPORTED;
  auto* n = new (std::nothrow) kerdock_mlp_s();
  if (n == nullptr) return KERDOCK_ERR_INVALID_ARG;
  n->in = in_dim;
  n->hid = hidden;
  n->out = out_dim;
  n->max_batch = max_batch;
  const int64_t sizes[6] = {int64_t(hidden) * in_dim, hidden, int64_t(hidden) * hidden,
                            hidden, int64_t(out_dim) * hidden, out_dim};
  n->off[0] = 0;
  for (int i = 0; i < 6; ++i) n->off[i + 1] = n->off[i] + sizes[i];
  n->count = n->off[6];
  const size_t P = size_t(n->count);
  n->state_bytes = 4 * a256(P * 4) + a256(size_t(sizes[0]) * 2) + a256(size_t(sizes[2]) * 2) +
                   a256(size_t(sizes[4]) * 2) + 256;
  const size_t B = size_t(max_batch);
  n->work_bytes = a256(B * in_dim * 2) + 2 * a256(B * hidden * 2) + a256(B * out_dim * 4) +
                  a256(B * out_dim * 2) + 2 * a256(B * hidden * 2);
  *mlp = n;
  return KERDOCK_OK;
}

int kerdock_mlp_set_input(kerdock_mlp_t mlp, int32_t mode) {
  if (mlp == nullptr || (mode != KERDOCK_MLP_INPUT_LINEAR && mode != KERDOCK_MLP_INPUT_ABS))
    return KERDOCK_ERR_INVALID_ARG;
  mlp->input_mode = mode;
  return KERDOCK_OK;
}

int kerdock_mlp_set_skip(kerdock_mlp_t mlp, float skip) {
  if (mlp == nullptr) return KERDOCK_ERR_INVALID_ARG;
  if (skip != 0.f && mlp->in != mlp->out) return KERDOCK_ERR_INVALID_ARG;
  mlp->skip = skip;
  return KERDOCK_OK;
}

int kerdock_mlp_sizes(kerdock_mlp_t mlp, size_t* state_bytes, size_t* work_bytes,
                      int64_t* param_count) {
  if (mlp == nullptr) return KERDOCK_ERR_INVALID_ARG;
  if (state_bytes) *state_bytes = mlp->state_bytes;
  if (work_bytes) *work_bytes = mlp->work_bytes;
  if (param_count) *param_count = mlp->count;
  return KERDOCK_OK;
}

int kerdock_mlp_bind(kerdock_mlp_t mlp, void* state_dev, size_t state_bytes, void* work_dev,
                     size_t work_bytes, void* stream) {
  if (mlp == nullptr || state_dev == nullptr || work_dev == nullptr) return KERDOCK_ERR_INVALID_ARG;
  kerdock_mlp_s* n = mlp;
  if (state_bytes < n->state_bytes || work_bytes < n->work_bytes) return KERDOCK_ERR_CAPACITY;
  if ((reinterpret_cast<uintptr_t>(state_dev) & 255) || (reinterpret_cast<uintptr_t>(work_dev) & 255))
    return KERDOCK_ERR_ALIGNMENT;
  const size_t P = size_t(n->count);
  char* s = static_cast<char*>(state_dev);
  n->master = reinterpret_cast<float*>(s);
  s += a256(P * 4);
  n->grads = reinterpret_cast<float*>(s);
  s += a256(P * 4);
  n->m = reinterpret_cast<float*>(s);
  s += a256(P * 4);
  n->v = reinterpret_cast<float*>(s);
  s += a256(P * 4);
  for (int w = 0; w < 3; ++w) {
    n->wbf[w] = reinterpret_cast<__nv_bfloat16*>(s);
    s += a256(size_t(n->off[2 * w + 1] - n->off[2 * w]) * 2);
  }
  n->loss = reinterpret_cast<float*>(s);
  const size_t B = size_t(n->max_batch);
  char* w = static_cast<char*>(work_dev);
  n->X0 = reinterpret_cast<__nv_bfloat16*>(w);
  w += a256(B * n->in * 2);
  n->H1 = reinterpret_cast<__nv_bfloat16*>(w);
  w += a256(B * n->hid * 2);
  n->H2 = reinterpret_cast<__nv_bfloat16*>(w);
  w += a256(B * n->hid * 2);
  n->Z = reinterpret_cast<float*>(w);
  w += a256(B * n->out * 4);
  n->dZ = reinterpret_cast<__nv_bfloat16*>(w);
  w += a256(B * n->out * 2);
  n->dH2 = reinterpret_cast<__nv_bfloat16*>(w);
  w += a256(B * n->hid * 2);
  n->dH1 = reinterpret_cast<__nv_bfloat16*>(w);
  n->stream = static_cast<cudaStream_t>(stream);
  n->bound = true;
  return KERDOCK_OK;
}

int kerdock_mlp_pointers(kerdock_mlp_t mlp, float** params, float** grads, int64_t* offsets) {
  if (mlp == nullptr || !mlp->bound) return KERDOCK_ERR_NOT_BOUND;
  if (params) *params = mlp->master;
  if (grads) *grads = mlp->grads;
  if (offsets)
    for (int i = 0; i < 7; ++i) offsets[i] = mlp->off[i];
  return KERDOCK_OK;
}

int kerdock_mlp_init(kerdock_mlp_t mlp, uint64_t seed) {
  if (mlp == nullptr) return KERDOCK_ERR_INVALID_ARG;
  kerdock_mlp_s* n = mlp;
  if (!n->bound) return KERDOCK_ERR_NOT_BOUND;
  // U(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases
  int64_t seg_end[6];
  float bound[6];
  const int fan[3] = {n->in, n->hid, n->hid};
  for (int i = 0; i < 6; ++i) {
    seg_end[i] = n->off[i + 1];
    bound[i] = (i % 2 == 0) ? 1.f / sqrtf(float(fan[i / 2])) : 0.f;
  }
  // the two small tables travel in the loss slot's neighbourhood: use the grads
  // buffer (overwritten by every backward) as a staging area
  int64_t* d_seg = reinterpret_cast<int64_t*>(n->grads);
  float* d_bound = reinterpret_cast<float*>(d_seg + 8);
  KD_CUDA_TRY(cudaMemcpyAsync(d_seg, seg_end, sizeof(seg_end), cudaMemcpyHostToDevice, n->stream));
  KD_CUDA_TRY(cudaMemcpyAsync(d_bound, bound, sizeof(bound), cudaMemcpyHostToDevice, n->stream));
  kd::init_kernel<<<kd::grid_for(n->count, 256), 256, 0, n->stream>>>(n->master, n->count, seed,
                                                                       d_seg, d_bound, 6);
  KD_CUDA_TRY(cudaGetLastError());
  KD_CUDA_TRY(cudaMemsetAsync(n->m, 0, size_t(n->count) * 4, n->stream));
  KD_CUDA_TRY(cudaMemsetAsync(n->v, 0, size_t(n->count) * 4, n->stream));
  KD_CUDA_TRY(cudaStreamSynchronize(n->stream));  // the staging tables are host locals
  for (int w = 0; w < 3; ++w) {
    const int64_t cnt = n->off[2 * w + 1] - n->off[2 * w];
    kd::f32_to_bf16_kernel<<<kd::grid_for(cnt, 256), 256, 0, n->stream>>>(
        n->master + n->off[2 * w], cnt, n->wbf[w]);
    KD_CUDA_TRY(cudaGetLastError());
  }
  n->step = 0;
  return KERDOCK_OK;
}

int kerdock_mlp_sync_weights(kerdock_mlp_t mlp) {
  if (mlp == nullptr || !mlp->bound) return KERDOCK_ERR_NOT_BOUND;
  for (int w = 0; w < 3; ++w) {
    const int64_t cnt = mlp->off[2 * w + 1] - mlp->off[2 * w];
    kd::f32_to_bf16_kernel<<<kd::grid_for(cnt, 256), 256, 0, mlp->stream>>>(
        mlp->master + mlp->off[2 * w], cnt, mlp->wbf[w]);
    KD_CUDA_TRY(cudaGetLastError());
  }
  return KERDOCK_OK;
}

int kerdock_mlp_forward(kerdock_mlp_t mlp, const float* feats, int32_t B, float feat_scale,
                        float* logits) {
  if (mlp == nullptr || feats == nullptr || logits == nullptr) return KERDOCK_ERR_INVALID_ARG;
  if (!mlp->bound) return KERDOCK_ERR_NOT_BOUND;
  if (B < 1 || B > mlp->max_batch) return KERDOCK_ERR_CAPACITY;
  return mlp_forward_impl(mlp, feats, B, feat_scale, logits);
}

int kerdock_mlp_backward(kerdock_mlp_t mlp, const float* feats, const float* labels, int32_t B,
                         float feat_scale, float pos_weight) {
  using namespace kd;
  if (mlp == nullptr || feats == nullptr || labels == nullptr) return KERDOCK_ERR_INVALID_ARG;
  kerdock_mlp_s* n = mlp;
  if (!n->bound) return KERDOCK_ERR_NOT_BOUND;
  if (B < 1 || B > n->max_batch) return KERDOCK_ERR_CAPACITY;
  int rc = mlp_forward_impl(n, feats, B, feat_scale, n->Z);
  if (rc != KERDOCK_OK) return rc;
  KD_CUDA_TRY(cudaMemsetAsync(n->loss, 0, sizeof(float), n->stream));
  const int64_t zc = int64_t(B) * n->out;
  bce_kernel<<<grid_for(zc, 256), 256, 0, n->stream>>>(n->Z, labels, zc, 1.f / float(B),
                                                        pos_weight, n->dZ, n->loss);
  KD_CUDA_TRY(cudaGetLastError());
  float* G = n->grads;
  GemmArgs g{};
  // dW3 = dZ^T H2, db3 = sum_b dZ
  g = GemmArgs{n->out, n->hid, B, n->dZ, 1, n->out, n->H2, 1, n->hid};
  rc = gemm(g, EpiF32{G + n->off[4], n->hid}, n->stream);
  if (rc != KERDOCK_OK) return rc;
  bias_grad_kernel<<<(n->out + 255) / 256, 256, 0, n->stream>>>(n->dZ, B, n->out, G + n->off[5]);
  // dH2 = (dZ W3) * [H2 > 0]
  g = GemmArgs{B, n->hid, n->out, n->dZ, n->out, 1, n->wbf[2], 1, n->hid};
  rc = gemm(g, EpiMaskBf16{n->H2, n->dH2, n->hid}, n->stream);
  if (rc != KERDOCK_OK) return rc;
  // dW2 = dH2^T H1, db2
  g = GemmArgs{n->hid, n->hid, B, n->dH2, 1, n->hid, n->H1, 1, n->hid};
  rc = gemm(g, EpiF32{G + n->off[2], n->hid}, n->stream);
  if (rc != KERDOCK_OK) return rc;
  bias_grad_kernel<<<(n->hid + 255) / 256, 256, 0, n->stream>>>(n->dH2, B, n->hid, G + n->off[3]);
  // dH1 = (dH2 W2) * [H1 > 0]
  g = GemmArgs{B, n->hid, n->hid, n->dH2, n->hid, 1, n->wbf[1], 1, n->hid};
  rc = gemm(g, EpiMaskBf16{n->H1, n->dH1, n->hid}, n->stream);
  if (rc != KERDOCK_OK) return rc;
  // dW1 = dH1^T X0, db1
  g = GemmArgs{n->hid, n->in, B, n->dH1, 1, n->hid, n->X0, 1, n->in};
  rc = gemm(g, EpiF32{G + n->off[0], n->in}, n->stream);
  if (rc != KERDOCK_OK) return rc;
  bias_grad_kernel<<<(n->hid + 255) / 256, 256, 0, n->stream>>>(n->dH1, B, n->hid, G + n->off[1]);
  KD_CUDA_TRY(cudaGetLastError());
  return KERDOCK_OK;
}

int kerdock_mlp_loss(kerdock_mlp_t mlp, float* loss_host) {
  if (mlp == nullptr || loss_host == nullptr) return KERDOCK_ERR_INVALID_ARG;
  if (!mlp->bound) return KERDOCK_ERR_NOT_BOUND;
  KD_CUDA_TRY(cudaMemcpyAsync(loss_host, mlp->loss, sizeof(float), cudaMemcpyDeviceToHost,
                              mlp->stream));
  KD_CUDA_TRY(cudaStreamSynchronize(mlp->stream));
  return KERDOCK_OK;
}

int kerdock_mlp_adamw(kerdock_mlp_t mlp, float lr, float beta1, float beta2, float eps,
                      float weight_decay) {
  if (mlp == nullptr) return KERDOCK_ERR_INVALID_ARG;
  kerdock_mlp_s* n = mlp;
  if (!n->bound) return KERDOCK_ERR_NOT_BOUND;
  n->step += 1;
  kd::AdamArgs a{};
  a.p = n->master;
  a.g = n->grads;
  a.m = n->m;
  a.v = n->v;
  a.count = n->count;
  a.lr = lr;
  a.beta1 = beta1;
  a.beta2 = beta2;
  a.eps = eps;
  a.wd = weight_decay;
  a.c1 = float(1.0 / (1.0 - std::pow(double(beta1), double(n->step))));
  a.c2 = float(1.0 / (1.0 - std::pow(double(beta2), double(n->step))));
  for (int w = 0; w < 3; ++w) {
    a.w_begin[w] = n->off[2 * w];
    a.w_end[w] = n->off[2 * w + 1];
    a.wbf[w] = n->wbf[w];
  }
  kd::adamw_kernel<<<kd::grid_for(n->count, 256), 256, 0, n->stream>>>(a);
  KD_CUDA_TRY(cudaGetLastError());
  return KERDOCK_OK;
}

int kerdock_mlp_destroy(kerdock_mlp_t mlp) {
  delete mlp;
  return KERDOCK_OK;
}

}  // extern "C"

extern "C" int kerdock_debug_gemm(const void* A, int64_t sAm, int64_t sAk, const void* B,
                                       int64_t sBn, int64_t sBk, int32_t M, int32_t N, int32_t K,
                                       int32_t kc, float* C, int64_t ldc, void* stream) {
  if (A == nullptr || B == nullptr || C == nullptr || M < 1 || N < 1 || K < 1 || ldc < N ||
      kc < 0 || kc % 64 != 0)
    return KERDOCK_ERR_INVALID_ARG;
  kd::GemmArgs g{M, N, K, static_cast<const __nv_bfloat16*>(A), sAm, sAk,
                 static_cast<const __nv_bfloat16*>(B), sBn, sBk};
  g.kc = kc >= K ? 0 : kc;
  return kd::gemm(g, kd::EpiF32{C, ldc, int64_t(M) * ldc}, static_cast<cudaStream_t>(stream));
}
