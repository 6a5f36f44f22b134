// preprocess.cu -- the preprocessing step of Algorithm 1 (Lemma 6).
//
// For every Kerdock basis b < d/2 and every row a_i of A the representation
// holds R[b][w][i] = sum_{p<n} (-1)^{Q_b(p) + w.p} A[i][p], i.e. the
// unnormalised Walsh-Hadamard transform (sqrt(d) H^{(x)k}, Lemma 6) of the
// sign-flipped, zero-padded row (Pi^* a_i)^T D_{M_b}.  The identity basis adds
// R[d/2][w][i] = sqrt(d) A[i][w] (zero for w >= n).
//
// Kernel design (d <= 1024): a CTA owns a tile of 32 rows of A, kept in
// shared memory across all the bases it processes, so A is read from HBM once.
// For each basis a warp g holds, per lane (= row), RG = d/NW consecutive p in
// registers: sign flip from the bit table, log2(RG) butterfly stages in
// registers; one shared-memory exchange then moves the NW warp-owned chunks
// into registers for the remaining log2(NW) stages and, at the same time,
// transposes the tile so that each store instruction of a warp writes 32
// consecutive i of one output row R[b][w][.] (128 B for float32).
#include "kerdock_internal.cuh"

namespace kd {
namespace {

constexpr int kTileRows = 32;

template <typename T>
__device__ __forceinline__ T to_out(float v);
template <>
__device__ __forceinline__ float to_out<float>(float v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 to_out<__nv_bfloat16>(float v) {
  return __float2bfloat16_rn(v);
}

// In-register unnormalised FWHT of length RG (bit h of the register index).
template <int RG>
__device__ __forceinline__ void fwht_regs(float (&v)[RG]) {
#pragma unroll
  for (int h = 1; h < RG; h <<= 1) {
#pragma unroll
    for (int r = 0; r < RG; ++r) {
      if (!(r & h)) {
        const float a = v[r], c = v[r + h];
        v[r] = a + c;
        v[r + h] = a - c;
      }
    }
  }
}

template <int LOG_D>
struct PreCfg {
  static constexpr int D = 1 << LOG_D;
  static constexpr int NW = LOG_D <= 2 ? 1 : LOG_D <= 4 ? 2 : LOG_D <= 6 ? 4 : 8;
  static constexpr int RG = D / NW;              // register values per thread in phase 1
  static constexpr int EXP = LOG_D >= 10 ? 2 : 1;  // exchange rounds (bounds shared memory)
  static constexpr int RGP = RG / EXP;           // registers exchanged per round
  static constexpr int AST = D + 4;              // A-tile row stride (floats): conflict-free LDS.128
  static constexpr int THREADS = NW * 32;
  static constexpr size_t SMEM =
      size_t(kTileRows) * AST * 4 + size_t(RGP) * NW * 32 * 4;
  static_assert(RGP >= NW, "phase 2 needs at least one w_lo per warp");
  static_assert(RG >= 4, "vector loads need 4 registers");
};

struct PreArgs {
  const float* A;
  int64_t lda, m, n;
  const uint32_t* signs;
  int64_t sign_words;
  void* R;
  int64_t ldr;
  int64_t num_tiles;
  int64_t items;  // num_tiles * (d/2 + 1)
};

template <int LOG_D, typename OutT>
__global__ void __launch_bounds__(PreCfg<LOG_D>::THREADS, 1)
    preprocess_small_kernel(const PreArgs a) {
  using C = PreCfg<LOG_D>;
  constexpr int D = C::D, NW = C::NW, RG = C::RG, RGP = C::RGP, AST = C::AST;
  constexpr int64_t B = D / 2 + 1;
  extern __shared__ __align__(16) float smem[];
  float* At = smem;                           // [32][AST]
  float* X = smem + size_t(kTileRows) * AST;  // [RGP * NW][32]
  OutT* R = static_cast<OutT*>(a.R);
  const int lane = threadIdx.x & 31;
  const int g = threadIdx.x >> 5;
  const float sqrt_d = float(1 << (LOG_D / 2));

  const int64_t per = a.items / gridDim.x, rem = a.items % gridDim.x;
  const int64_t beg = blockIdx.x * per + (blockIdx.x < rem ? blockIdx.x : rem);
  const int64_t end = beg + per + (blockIdx.x < rem ? 1 : 0);
  int64_t cur_tile = -1;

  for (int64_t item = beg; item < end; ++item) {
    const int64_t t = item / B;
    const int b = int(item - t * B);
    const int64_t i0 = t * kTileRows;
    if (t != cur_tile) {
      __syncthreads();  // everyone is done with the previous tile
      for (int idx = threadIdx.x; idx < kTileRows * D; idx += C::THREADS) {
        const int i = idx / D, p = idx % D;
        float v = 0.f;
        if (i0 + i < a.m && p < a.n) v = a.A[(i0 + i) * a.lda + p];
        At[i * AST + p] = v;
      }
      __syncthreads();
      cur_tile = t;
    }
    const bool ident = b == D / 2;

    // Phase 1: lane = row i, registers = p in [g*RG, (g+1)*RG).
    float v[RG];
#pragma unroll
    for (int r = 0; r < RG; r += 4) {
      const float4 q = *reinterpret_cast<const float4*>(&At[lane * AST + g * RG + r]);
      v[r] = q.x;
      v[r + 1] = q.y;
      v[r + 2] = q.z;
      v[r + 3] = q.w;
    }
    if (!ident) {
      const uint32_t* srow = a.signs + int64_t(b) * a.sign_words;
      if constexpr (RG >= 32) {
#pragma unroll
        for (int r0 = 0; r0 < RG; r0 += 32) {
          const uint32_t word = __ldg(srow + (g * RG + r0) / 32);
#pragma unroll
          for (int r = 0; r < 32; ++r) v[r0 + r] = flip_sign(v[r0 + r], (word >> r) & 1u);
        }
      } else {
        const uint32_t word = __ldg(srow + (g * RG) / 32) >> ((g * RG) & 31);
#pragma unroll
        for (int r = 0; r < RG; ++r) v[r] = flip_sign(v[r], (word >> r) & 1u);
      }
      fwht_regs<RG>(v);
    }

    // Exchange + phase 2, in EXP rounds over the top register bit(s).
#pragma unroll
    for (int part = 0; part < C::EXP; ++part) {
      __syncthreads();  // X is free
#pragma unroll
      for (int r = 0; r < RGP; ++r) X[(g * RGP + r) * 32 + lane] = v[part * RGP + r];
      __syncthreads();
#pragma unroll
      for (int u = 0; u < RGP / NW; ++u) {
        const int wl = g * (RGP / NW) + u;
        float y[NW];
#pragma unroll
        for (int h = 0; h < NW; ++h) y[h] = X[(h * RGP + wl) * 32 + lane];
        if (!ident) {
          fwht_regs<NW>(y);
        } else {
#pragma unroll
          for (int h = 0; h < NW; ++h) y[h] *= sqrt_d;
        }
        if (i0 + lane < a.ldr) {
#pragma unroll
          for (int h = 0; h < NW; ++h) {
            const int64_t w = int64_t(h) * RG + part * RGP + wl;
            R[(int64_t(b) * D + w) * a.ldr + i0 + lane] = to_out<OutT>(y[h]);
          }
        }
      }
    }
  }
}

template <int LOG_D, typename OutT>
int launch_small(const Plan& p) {
  using C = PreCfg<LOG_D>;
  auto kern = preprocess_small_kernel<LOG_D, OutT>;
  KD_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   int(C::SMEM)));
  int occ = 0;
  KD_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, C::THREADS, C::SMEM));
  if (occ < 1) return KERDOCK_ERR_UNSUPPORTED;
  PreArgs a;
  a.A = p.A;
  a.lda = p.lda;
  a.m = p.m;
  a.n = p.n;
  a.signs = p.signs();
  a.sign_words = p.sign_words;
  a.R = p.repr;
  a.ldr = p.ldr;
  a.num_tiles = (p.ldr + kTileRows - 1) / kTileRows;
  a.items = a.num_tiles * p.B;
  int64_t grid = int64_t(p.num_sms) * occ;
  if (grid > a.items) grid = a.items;
  kern<<<unsigned(grid), C::THREADS, C::SMEM, p.stream>>>(a);
  KD_CUDA_TRY(cudaGetLastError());
  return KERDOCK_OK;
}

template <typename OutT>
int launch_typed(const Plan& p) {
  switch (p.k) {
    case 2: return launch_small<2, OutT>(p);
    case 4: return launch_small<4, OutT>(p);
    case 6: return launch_small<6, OutT>(p);
    case 8: return launch_small<8, OutT>(p);
    case 10: return launch_small<10, OutT>(p);
    default: return KERDOCK_ERR_UNSUPPORTED;
  }
}

}  // namespace

int launch_preprocess(const Plan& p) {
  return p.dtype == KERDOCK_BF16 ? launch_typed<__nv_bfloat16>(p) : launch_typed<float>(p);
}

}  // namespace kd
