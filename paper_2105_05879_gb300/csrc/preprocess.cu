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
// Per basis the sign bits become float sign masks in shared memory (one XOR
// per element).  Phase 1: a warp g holds, per lane (= row), RG = d/NW
// consecutive p in registers as float pairs and runs log2(RG) butterfly
// stages (packed add/sub.f32x2).  One shared-memory exchange then moves the
// NW warp-owned chunks so that each thread holds two rows x two adjacent w
// for the remaining log2(NW) stages (packed across the two rows), and stores
// 8-byte row pairs: a warp store writes two 128-byte runs of consecutive i of
// output rows R[b][w][.] (float32).
#include "kerdock_internal.cuh"

namespace kd {
namespace {

constexpr int kTileRows = 32;

// Packed-pair helpers: two float lanes in one 64-bit register (add/sub.f32x2).
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;"
      : "=l"(r)
      : "l"(*reinterpret_cast<unsigned long long*>(&a)),
        "l"(*reinterpret_cast<unsigned long long*>(&b)));
  return *reinterpret_cast<float2*>(&r);
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;"
      : "=l"(r)
      : "l"(*reinterpret_cast<unsigned long long*>(&a)),
        "l"(*reinterpret_cast<unsigned long long*>(&b)));
  return *reinterpret_cast<float2*>(&r);
}

// Unnormalised FWHT of length 2*NP held as NP float2 pairs (element 2i and
// 2i+1 in pair i): the stride-1 stage is done inside each pair, the other
// stages on whole pairs with packed adds.
template <int NP>
__device__ __forceinline__ void fwht_pairs(float2 (&v)[NP]) {
#pragma unroll
  for (int i = 0; i < NP; ++i) v[i] = make_float2(v[i].x + v[i].y, v[i].x - v[i].y);
#pragma unroll
  for (int h = 1; h < NP; h <<= 1) {
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      if (!(i & h)) {
        const float2 a = v[i], c = v[i + h];
        v[i] = add2(a, c);
        v[i + h] = sub2(a, c);
      }
    }
  }
}

// Unnormalised FWHT of length NH over an array of float2, each pair carrying
// two independent transforms (two rows).
template <int NH>
__device__ __forceinline__ void fwht_across(float2 (&v)[NH]) {
#pragma unroll
  for (int h = 1; h < NH; h <<= 1) {
#pragma unroll
    for (int i = 0; i < NH; ++i) {
      if (!(i & h)) {
        const float2 a = v[i], c = v[i + h];
        v[i] = add2(a, c);
        v[i + h] = sub2(a, c);
      }
    }
  }
}

template <typename T>
__device__ __forceinline__ void store_pair(T* dst, float2 v);
template <>
__device__ __forceinline__ void store_pair<float>(float* dst, float2 v) {
  *reinterpret_cast<float2*>(dst) = v;
}
template <>
__device__ __forceinline__ void store_pair<__nv_bfloat16>(__nv_bfloat16* dst, float2 v) {
  *reinterpret_cast<__nv_bfloat162*>(dst) = __floats2bfloat162_rn(v.x, v.y);
}

template <int LOG_D>
struct PreCfg {
  static constexpr int D = 1 << LOG_D;
  static constexpr int NW = LOG_D <= 2 ? 1 : LOG_D <= 4 ? 2 : LOG_D <= 6 ? 4 : 8;
  static constexpr int RG = D / NW;                // phase-1 values per thread
  static constexpr int EXP = LOG_D >= 10 ? 2 : 1;  // exchange rounds (bounds shared memory)
  static constexpr int RGP = RG / EXP;             // values exchanged per round
  static constexpr int WPAIRS = RGP / 2 / (2 * NW);  // phase-2 w pairs per thread per round
  static constexpr int AST = D + 4;                // A-tile row stride (floats): conflict-free LDS.128
  static constexpr int THREADS = NW * 32;
  static constexpr size_t SMEM = size_t(kTileRows) * AST * 4 + size_t(RGP) * NW * 32 * 4 +
                                 size_t(D > 32 ? D : 32) * 4;
  static_assert(WPAIRS >= 1, "phase 2 needs at least one w pair per thread");
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
  float* At = smem;                                         // [32][AST]
  float2* X2 = reinterpret_cast<float2*>(smem + size_t(kTileRows) * AST);  // [RGP*NW/2][32]
  uint32_t* Msk = reinterpret_cast<uint32_t*>(smem + size_t(kTileRows) * AST +
                                              size_t(RGP) * NW * 32);     // [D] sign masks
  OutT* R = static_cast<OutT*>(a.R);
  const int lane = threadIdx.x & 31;
  const int g = threadIdx.x >> 5;
  const int rp = lane & 15, wsel = lane >> 4;  // phase-2 roles: row pair, w-pair selector
  const float sqrt_d = float(1 << (LOG_D / 2));

  const int64_t per = a.items / gridDim.x, rem = a.items % gridDim.x;
  const int64_t beg = blockIdx.x * per + (blockIdx.x < rem ? blockIdx.x : rem);
  const int64_t end = beg + per + (blockIdx.x < rem ? 1 : 0);
  int64_t cur_tile = -1;

  for (int64_t item = beg; item < end; ++item) {
    const int64_t t = item / B;
    const int b = int(item - t * B);
    const int64_t i0 = t * kTileRows;
    const bool ident = b == D / 2;
    __syncthreads();  // everyone is done with the previous item (tile, masks, exchange)
    if (t != cur_tile) {
      for (int idx = threadIdx.x; idx < kTileRows * D; idx += C::THREADS) {
        const int i = idx / D, p = idx % D;
        float v = 0.f;
        if (i0 + i < a.m && p < a.n) v = a.A[(i0 + i) * a.lda + p];
        At[i * AST + p] = v;
      }
      cur_tile = t;
    }
    if (!ident) {  // step (i) of Lemma 6 as float sign masks for this basis
      const uint32_t* srow = a.signs + int64_t(b) * a.sign_words;
      for (int p = threadIdx.x; p < D; p += C::THREADS)
        Msk[p] = ((__ldg(srow + (p >> 5)) >> (p & 31)) & 1u) << 31;
    }
    __syncthreads();

    // Phase 1: lane = row i, registers = p in [g*RG, (g+1)*RG) as pairs.
    float2 v[RG / 2];
#pragma unroll
    for (int r = 0; r < RG; r += 4) {
      float4 q = *reinterpret_cast<const float4*>(&At[lane * AST + g * RG + r]);
      if (!ident) {
        const uint4 mk = *reinterpret_cast<const uint4*>(&Msk[g * RG + r]);
        q.x = __uint_as_float(__float_as_uint(q.x) ^ mk.x);
        q.y = __uint_as_float(__float_as_uint(q.y) ^ mk.y);
        q.z = __uint_as_float(__float_as_uint(q.z) ^ mk.z);
        q.w = __uint_as_float(__float_as_uint(q.w) ^ mk.w);
      }
      v[r / 2] = make_float2(q.x, q.y);
      v[r / 2 + 1] = make_float2(q.z, q.w);
    }
    if (!ident) fwht_pairs<RG / 2>(v);

    // Exchange + phase 2, in EXP rounds over the top register bit(s).  The
    // exchange layout is [w/2][row][2] so that phase 1 writes 8 bytes per
    // value pair and phase 2 reads 16 bytes = two rows x two adjacent w.
#pragma unroll
    for (int part = 0; part < C::EXP; ++part) {
      if (part > 0) __syncthreads();  // X is free
#pragma unroll
      for (int r2 = 0; r2 < RGP / 2; ++r2) X2[(g * (RGP / 2) + r2) * 32 + lane] = v[part * (RGP / 2) + r2];
      __syncthreads();
#pragma unroll
      for (int u = 0; u < C::WPAIRS; ++u) {
        const int wp = (g * 2 + wsel) * C::WPAIRS + u;  // w pair index within the round
        float2 ye[NW], yo[NW];  // (row 2rp, row 2rp+1) for w_lo = 2wp and 2wp+1
#pragma unroll
        for (int h = 0; h < NW; ++h) {
          const float4 f = *reinterpret_cast<const float4*>(&X2[(h * (RGP / 2) + wp) * 32 + 2 * rp]);
          ye[h] = make_float2(f.x, f.z);
          yo[h] = make_float2(f.y, f.w);
        }
        if (!ident) {
          fwht_across<NW>(ye);
          fwht_across<NW>(yo);
        } else {
#pragma unroll
          for (int h = 0; h < NW; ++h) {
            ye[h] = make_float2(ye[h].x * sqrt_d, ye[h].y * sqrt_d);
            yo[h] = make_float2(yo[h].x * sqrt_d, yo[h].y * sqrt_d);
          }
        }
        const int64_t row = i0 + 2 * rp;
        if (row < a.ldr) {
#pragma unroll
          for (int h = 0; h < NW; ++h) {
            const int64_t w = int64_t(h) * RG + part * RGP + 2 * wp;
            store_pair<OutT>(R + (int64_t(b) * D + w) * a.ldr + row, ye[h]);
            store_pair<OutT>(R + (int64_t(b) * D + w + 1) * a.ldr + row, yo[h]);
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
