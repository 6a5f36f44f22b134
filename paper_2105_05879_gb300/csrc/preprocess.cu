// preprocess.cu -- the preprocessing step of Algorithm 1 (Lemma 6).
//
// For every Kerdock basis b < d/2 and every row a_i of A the representation
// holds R[b][w][i] = sum_{p<n} (-1)^{Q_b(p) + w.p} A[i][p], i.e. the
// unnormalised Walsh-Hadamard transform (sqrt(d) H^{(x)k}, Lemma 6) of the
// sign-flipped, zero-padded row (Pi^* a_i)^T D_{M_b}.  The identity basis adds
// R[d/2][w][i] = sqrt(d) A[i][w] (zero for w >= n).
//
// Kernels:
//  * d = 1024 (preprocess_d1024_kernel): as below, but the 16-row tile of A
//    sits in tensor memory (each thread's 64 words in its own lane), a thread
//    transforms a row pair in phase 1 (one sign bit flips both rows) and one
//    exchange of 8-byte row pairs replaces two rounds of 4-byte words.
//  * d <= 256 (preprocess_small_kernel): a CTA owns a tile of 16 rows of A,
//    kept in shared memory across all the bases it processes, so A is read
//    from HBM once.  Per basis each thread flips the signs of its p range from
//    its own sign words (one shift and one XOR per element).  Phase 1: a
//    thread (row, source) holds RG consecutive p in registers as float pairs
//    and runs log2(RG) butterfly stages (packed add/sub.f32x2).  One
//    shared-memory exchange then moves the sources so that each thread holds
//    two rows x one w for the remaining stages (packed across the two rows),
//    and stores 8-byte row pairs (streaming stores).  Groups of 16 CTAs own
//    adjacent tiles and walk the bases in step, so every 128-byte line of an
//    output row R[b][w][.] is completed by two CTAs at about the same time.
//  * d = 1024, bfloat16 (preprocess_d1024_tc_kernel): W_16 (x) W_16 (x) W_4 on
//    the tensor cores, 64-row tiles.
//  * d = 4096, bfloat16 (preprocess_d4096_tc_kernel, precision form) and
//    float32 (preprocess_d4096_tc32_kernel): the three 16-point stages of
//    W_16 (x) W_16 (x) W_16 on the tensor cores, float32 as float16 hi + lo
//    operand pairs.
#include <cuda.h>  // CUtensorMap (types only; the encoder comes from the runtime)

#include <cuda_fp16.h>

#include <type_traits>

#include "kerdock_internal.cuh"

namespace kd {
namespace {

constexpr int kTileRows = 16;

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
// Streaming (evict-first) stores: the representation is written once here and
// read back only by later queries, long after it has left L2.
template <>
__device__ __forceinline__ void store_pair<float>(float* dst, float2 v) {
  asm volatile("st.global.cs.v2.f32 [%0], {%1, %2};" ::"l"(dst), "f"(v.x), "f"(v.y) : "memory");
}
template <>
__device__ __forceinline__ void store_pair<__nv_bfloat16>(__nv_bfloat16* dst, float2 v) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
  asm volatile("st.global.cs.b32 [%0], %1;" ::"l"(dst),
               "r"(*reinterpret_cast<const uint32_t*>(&h))
               : "memory");
}

// Per-size configuration.  A CTA owns TI = 16 rows; D = NW * 2^LH * RG with
// NW warps, 2^LH lane halves and RG phase-1 registers per thread; SRC = D/RG
// sources are combined in phase 2; EXP exchange rounds bound shared memory.
template <int LOG_D>
struct PreCfg {
  static constexpr int D = 1 << LOG_D;
  static constexpr int NW = LOG_D >= 10 ? 8 : LOG_D >= 8 ? 4 : LOG_D >= 6 ? 2 : 1;
  static constexpr int LH = LOG_D >= 4 ? 1 : 0;
  static constexpr int RG = D / (NW << LH);
  static constexpr int SRC = D / RG;
  static constexpr int EXP = LOG_D >= 10 ? 2 : 1;
  static constexpr int RGP = RG / EXP;
  static constexpr int WPS = RGP / (4 * NW);  // phase-2 w per thread per round
  static constexpr int AST = D + 4;            // A-tile row stride (floats): conflict-free LDS.128
  static constexpr int XST = RGP * kTileRows + 16;  // floats per source in X (bank shift 16)
  static constexpr int THREADS = NW * 32;
  static constexpr size_t SMEM = size_t(kTileRows) * AST * 4 + size_t(SRC) * XST * 4;
  static_assert(WPS >= 1, "phase 2 needs at least one w per thread");
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
  int64_t group;  // G: consecutive CTAs (or clusters) that sweep the bases in step
  uint32_t* status;  // the plan's device status word
  int* work;         // per-tile counters of the dynamic schedule (zeroed before the launch)
};

// Work split.  Tiles are taken in groups of G adjacent tiles; the G CTAs (or
// clusters) of a group own one tile each and walk the same range of (tile
// group, basis) items, so that at any time the group writes G adjacent row
// segments of every output row R[b][w][.] and L2 receives whole 128-byte
// lines instead of isolated 32- or 64-byte pieces.  Within a CTA the items are
// tile-major, so the A tile in shared memory is reloaded only when the tile
// changes.
struct ItemRange {
  int64_t beg, end, slot;
};
__device__ __forceinline__ ItemRange item_range(int64_t unit, int64_t units, int64_t group,
                                                int64_t num_tiles, int64_t B) {
  const int64_t ngrp = units / group, grp = unit / group;
  const int64_t ntg = (num_tiles + group - 1) / group;
  const int64_t items = ntg * B;
  const int64_t per = items / ngrp, rem = items % ngrp;
  ItemRange r;
  r.beg = grp * per + (grp < rem ? grp : rem);
  r.end = r.beg + per + (grp < rem ? 1 : 0);
  r.slot = unit % group;
  // a slot past the last tile has nothing to do in the last tile group, which
  // is the tail of the item space
  if ((ntg - 1) * group + r.slot >= num_tiles) {
    const int64_t lim = (ntg - 1) * B;
    if (r.end > lim) r.end = lim;
    if (r.beg > r.end) r.beg = r.end;
  }
  return r;
}

template <int LOG_D, typename OutT>
__global__ void __launch_bounds__(PreCfg<LOG_D>::THREADS, 2)
    preprocess_small_kernel(const PreArgs a) {
  using C = PreCfg<LOG_D>;
  constexpr int D = C::D, RG = C::RG, RGP = C::RGP, AST = C::AST, SRC = C::SRC;
  constexpr int XST = C::XST;
  constexpr int NWD = RG >= 32 ? RG / 32 : 1;  // sign words per phase-1 thread
  constexpr int64_t B = D / 2 + 1;
  extern __shared__ __align__(16) float smem[];
  float* At = smem;                                 // [16][AST]
  float* X = smem + size_t(kTileRows) * AST;        // [SRC][XST]: [w][row] per source
  OutT* R = static_cast<OutT*>(a.R);
  const int lane = threadIdx.x & 31;
  const int g = threadIdx.x >> 5;
  const int row = lane & 15, hb = lane >> 4;             // phase 1: row, lane half
  const int src = (g << C::LH) + hb;                     // phase-1 source index
  const bool p1 = C::LH == 1 || hb == 0;                 // lane takes part in phase 1
  const int rp = lane & 7, wsel = lane >> 3;             // phase 2: row pair, w selector
  const float sqrt_d = float(1 << (LOG_D / 2));

  const ItemRange ir = item_range(blockIdx.x, gridDim.x, a.group, a.num_tiles, B);
  const int64_t beg = ir.beg, end = ir.end;
  int64_t cur_tile = -1;

  for (int64_t item = beg; item < end; ++item) {
    const int64_t tg = item / B;
    const int b = int(item - tg * B);
    const int64_t t = tg * a.group + ir.slot;
    const int64_t i0 = t * kTileRows;
    const bool ident = b == D / 2;
    __syncthreads();  // everyone is done with the previous item's tile and exchange
    if (t != cur_tile) {
      for (int idx = threadIdx.x; idx < kTileRows * D; idx += C::THREADS) {
        const int i = idx / D, p = idx % D;
        float v = 0.f;
        if (i0 + i < a.m && p < a.n) v = a.A[(i0 + i) * a.lda + p];
        At[i * AST + p] = v;
      }
      cur_tile = t;
    }
    // Sign bits of this thread's p range [src*RG, (src+1)*RG) (step (i) of
    // Lemma 6), shifted down to bit 0 when RG < 32.
    uint32_t wcur[NWD];
    {
      const uint32_t* srow = a.signs + int64_t(b < D / 2 ? b : 0) * a.sign_words;
      if (RG >= 32) {
#pragma unroll
        for (int c = 0; c < NWD; ++c) wcur[c] = p1 ? __ldg(srow + src * NWD + c) : 0u;
      } else {
        const int p0 = src * RG;
        wcur[0] = p1 ? __ldg(srow + (p0 >> 5)) >> (p0 & 31) : 0u;
      }
    }
    __syncthreads();

    // Phase 1: lane = (row, half), registers = p in [src*RG, (src+1)*RG) as
    // pairs; the sign flip XORs bit r of the thread's sign words into the
    // float sign bit.
    float2 v[RG / 2];
    if (p1) {
#pragma unroll
      for (int r = 0; r < RG; r += 4) {
        float4 q = *reinterpret_cast<const float4*>(&At[row * AST + src * RG + r]);
        if (!ident) {
          uint32_t f[4];
#pragma unroll
          for (int e = 0; e < 4; ++e)
            f[e] = (wcur[(r + e) >> 5] << (31 - ((r + e) & 31))) & 0x80000000u;
          q.x = __uint_as_float(__float_as_uint(q.x) ^ f[0]);
          q.y = __uint_as_float(__float_as_uint(q.y) ^ f[1]);
          q.z = __uint_as_float(__float_as_uint(q.z) ^ f[2]);
          q.w = __uint_as_float(__float_as_uint(q.w) ^ f[3]);
        }
        v[r / 2] = make_float2(q.x, q.y);
        v[r / 2 + 1] = make_float2(q.z, q.w);
      }
      if (!ident) fwht_pairs<RG / 2>(v);
    }

    // Exchange ([source][w][row]) + phase 2 in EXP rounds over the top register bit(s).
#pragma unroll
    for (int part = 0; part < C::EXP; ++part) {
      if (part > 0) __syncthreads();  // X is free
      if (p1) {
#pragma unroll
        for (int r2 = 0; r2 < RGP / 2; ++r2) {
          const float2 val = v[part * (RGP / 2) + r2];
          X[src * XST + (2 * r2) * kTileRows + row] = val.x;
          X[src * XST + (2 * r2 + 1) * kTileRows + row] = val.y;
        }
      }
      __syncthreads();
#pragma unroll
      for (int u = 0; u < C::WPS; ++u) {
        const int wl = (g * 4 + wsel) * C::WPS + u;  // w within the round's block
        float2 y[SRC];  // (row 2rp, row 2rp+1)
#pragma unroll
        for (int h = 0; h < SRC; ++h)
          y[h] = *reinterpret_cast<const float2*>(&X[h * XST + wl * kTileRows + 2 * rp]);
        if (!ident) {
          fwht_across<SRC>(y);
        } else {
#pragma unroll
          for (int h = 0; h < SRC; ++h) y[h] = make_float2(y[h].x * sqrt_d, y[h].y * sqrt_d);
        }
        const int64_t orow = i0 + 2 * rp;
        if (orow < a.ldr) {
          // output w = h * RG + part * RGP + wl for source h
          OutT* rb = R + (int64_t(b) * D + part * RGP + wl) * a.ldr + orow;
#pragma unroll
          for (int h = 0; h < SRC; ++h) store_pair<OutT>(rb + int64_t(h) * RG * a.ldr, y[h]);
        }
      }
    }
  }
}

// Largest power of two <= limit and <= num_tiles (the tile group size G).
int64_t pick_group(int64_t num_tiles, int64_t limit) {
  int64_t g = 1;
  while (g * 2 <= limit && g * 2 <= num_tiles) g *= 2;
  return g;
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
  a.status = p.status();
  a.num_tiles = (p.ldr + kTileRows - 1) / kTileRows;
  // groups of up to 16 CTAs on adjacent 16-row tiles (256 consecutive rows)
  a.group = pick_group(a.num_tiles, 16);
  int64_t ngrp = int64_t(p.num_sms) * occ / a.group;
  const int64_t items = ((a.num_tiles + a.group - 1) / a.group) * p.B;
  if (ngrp > items) ngrp = items;
  if (ngrp < 1) ngrp = 1;
  kern<<<unsigned(ngrp * a.group), C::THREADS, C::SMEM, p.stream>>>(a);
  KD_CUDA_TRY(cudaGetLastError());
  return KERDOCK_OK;
}


// ---------------------------------------------------------------------------
// Precision form, d = 4096, bfloat16 representation: the three 16-point
// stages of W_4096 = W_16 (x) W_16 (x) W_16 on the tensor cores
// (mma.sync m16n8k16, float16 operands, float32 accumulation).  Write
// p = 256 p2 + 16 p1 + p0 and w = 256 w2 + 16 w1 + w0.  For one row and one
// p2, stage 1 multiplies W_16 by the 16 x 16 block [p0][p1] (two n-tiles of
// 8 p1) and gives [w0][p1]; its accumulator fragments are exactly the B
// fragments of stage 2 over p1 (the C layout's columns are B's k), which gives
// [w1][w0].  That block goes to shared memory (stmatrix) as E[row][w1][p2][w0];
// stage 3 reads 16 p2 x 16 w0 per (row, w1) back with ldmatrix.trans, multiplies
// by W_16 and gives [w2][w0]; eight rows of one w1 are packed as row pairs
// into F[w2][w0][row] (32-byte rows, 32-byte swizzle) and written with one
// 4-D TMA store (16 rows x 16 w0 x 16 w2).  The CTA's 16-row tile of A sits
// in tensor memory (128 KiB) as float16, each row scaled by a power of two
// 2^e_r that brings its largest entry into [1/2, 1), laid out so that each
// thread's words for one (row, p2) are four consecutive columns of its own
// lane; stage 3's A operand is W_16 2^-e_r (exact in float16), so the output
// comes back at A's scale.  Float16 keeps 11 significant bits: the input and
// the two intermediate stages each add ~2^-12 ||a_i|| (rms over w) beside the
// final bfloat16 rounding; the identity basis uses 4 I in all three stages
// (x 64 = sqrt(d)).
// ---------------------------------------------------------------------------
namespace tc {

constexpr int TI = 16, WARPS = 16, THREADS = WARPS * 32, D = 4096;
constexpr int E_W1 = 16 * 32 + 16;           // bytes per (row, w1): 16 p2 x 32 B + pad
constexpr int E_ROW = 16 * E_W1;             // bytes per row
constexpr int E_BYTES = TI * E_ROW;          // 135168
constexpr int F_WARP = 16 * 8 * TI * 2;      // [w2][w0 half][row] bfloat16 per warp: 4 KiB
constexpr size_t OFF_SLOT = size_t(E_BYTES) + size_t(WARPS) * F_WARP;
constexpr size_t OFF_RFRAG = OFF_SLOT + 16;                 // [2][TI rows][32 lanes] uint4
constexpr size_t OFF_RMAX = OFF_RFRAG + 2 * size_t(TI) * 32 * 16;
constexpr size_t OFF_REM = OFF_RMAX + TI * 4;
constexpr size_t OFF_REXP = OFF_REM + TI * 4;
constexpr size_t SMEM = OFF_REXP + TI * 4;
constexpr uint32_t TMEM_COLS = 256;          // 4 rows x 16 p2 x 4 words per lane

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&h);
}
__device__ __forceinline__ uint32_t pack_f16x2(float lo, float hi) {
  const __half2 h = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&h);
}
// float16 bits of 2^k, exact for k in [-24, 15]
__device__ __forceinline__ uint32_t f16_pow2(int k) {
  return k >= -14 ? uint32_t(k + 15) << 10 : 1u << (k + 24);
}
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%10,%10,%10,%10};"
      : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1), "f"(0.f));
}
__device__ __forceinline__ void stmatrix_x4(uint32_t addr, uint32_t e0, uint32_t e1, uint32_t e2,
                                            uint32_t e3) {
  asm volatile("stmatrix.sync.aligned.m8n8.x4.shared.b16 [%0], {%1, %2, %3, %4};" ::"r"(addr),
               "r"(e0), "r"(e1), "r"(e2), "r"(e3)
               : "memory");
}
__device__ __forceinline__ void ldmatrix_x2_trans(uint32_t addr, uint32_t (&m)[2]) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0, %1}, [%2];"
               : "=r"(m[0]), "=r"(m[1])
               : "r"(addr)
               : "memory");
}
// Loads are asynchronous: the registers are valid after tmem_wait_ld, which
// names them so that the compiler does not read them earlier.
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t (&v)[4]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
               : "r"(taddr)
               : "memory");
}
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&u)[4], uint32_t (&v)[4]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(u[0]), "+r"(u[1]), "+r"(u[2]), "+r"(u[3]), "+r"(v[0]), "+r"(v[1]),
                 "+r"(v[2]), "+r"(v[3])
               :
               : "memory");
}
__device__ __forceinline__ void tmem_st4(uint32_t taddr, const uint32_t (&v)[4]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr),
               "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3])
               : "memory");
}
__device__ __forceinline__ void tma_store_4d(const CUtensorMap* map, uint32_t src, int c0, int c1,
                                             int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%1, %2, %3, %4}], [%5];" ::"l"(
          reinterpret_cast<uint64_t>(map)),
      "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(src)
      : "memory");
}

// Column of tensor memory holding a thread's four words for (row slot rl, p2).
__device__ __forceinline__ uint32_t tcol(int rl, int p2) { return uint32_t((rl * 16 + p2) * 4); }

__global__ void __launch_bounds__(THREADS, 1)
    preprocess_d4096_tc_kernel(const PreArgs a, const __grid_constant__ CUtensorMap tmap) {
  constexpr int64_t B = D / 2 + 1;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* E = smem;
  unsigned char* Fw = smem + E_BYTES + (threadIdx.x >> 5) * F_WARP;  // this warp's F
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + OFF_SLOT);
  uint4* rfrag = reinterpret_cast<uint4*>(smem + OFF_RFRAG);     // [W16 | 4 I][row][lane]
  uint32_t* rmax = reinterpret_cast<uint32_t*>(smem + OFF_RMAX);  // row maxima (float bits)
  int* rrem = reinterpret_cast<int*>(smem + OFF_REM);             // exponent left for float32
  int* rexp = reinterpret_cast<int*>(smem + OFF_REXP);            // row scale exponents e_r
  uint32_t smask = 0u;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, q = lane & 3;
  const int quarter = warp & 3, pq = warp >> 2;  // lane quarter of tensor memory; p2 quarter
  const bool aligned = (smem_addr(smem) & 1023u) == 0;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(tmem_slot);
  const uint32_t tlane = tmem + (uint32_t(quarter * 32) << 16);
  if (tid == 0 && !aligned) set_status(a.status, kStatusBadIndex);

  // A fragments (rows g, g+8; columns 2q, 2q+1, 2q+8, 2q+9) of W_16 and of 4 I.
  uint32_t aw[4], ai[4];
  {
    const int rr[4] = {g, g + 8, g, g + 8};
    const int cc[4] = {2 * q, 2 * q, 2 * q + 8, 2 * q + 8};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float w0 = (__popc(rr[e] & cc[e]) & 1) ? -1.f : 1.f;
      const float w1 = (__popc(rr[e] & (cc[e] + 1)) & 1) ? -1.f : 1.f;
      aw[e] = pack_f16x2(w0, w1);
      ai[e] = pack_f16x2(rr[e] == cc[e] ? 4.f : 0.f, rr[e] == cc[e] + 1 ? 4.f : 0.f);
    }
  }

  const ItemRange ir = item_range(blockIdx.x, gridDim.x, a.group, a.num_tiles, B);
  // Step (i) of Lemma 6 in registers.  The B fragment word j of (p2, lane)
  // holds p = 256 p2 + 16 (g + 8 (j >> 1)) + 2q + 8 (j & 1) and p + 1, so the
  // warp's p2 quarter needs two sign words per p2 (j >> 1 = 0, 1), both at bit
  // offset 16 (g & 1) + 2q, plus 8 for j & 1.  They are requested for the next
  // basis while stage 3 of this one runs.
  const int wsh = 16 * (g & 1) + 2 * q;
  auto load_words = [&](int b, uint32_t (&wd)[8]) {
    const uint32_t* srow =
        a.signs + int64_t(b == D / 2 ? 0 : b) * a.sign_words + 32 * pq + (g >> 1);
#pragma unroll
    for (int k = 0; k < 8; ++k)
      wd[k] = b == D / 2 ? 0u : __ldg(srow + 8 * (k >> 1) + 4 * (k & 1)) >> wsh;
  };
  uint32_t wd[8];
  if (ir.beg < ir.end) load_words(int(ir.beg % B), wd);
  int64_t cur_tile = -1;
  for (int64_t item = ir.beg; item < ir.end; ++item) {
    const int64_t tg = item / B;
    const int b = int(item - tg * B);
    const int64_t t = tg * a.group + ir.slot;
    const int64_t i0 = t * TI;
    const bool ident = b == D / 2;

    if (t != cur_tile) {  // this warp's share of the tile into its lanes of tensor memory
      // A row whose largest entry lies in [2^-8, 2^6) is used as it is: its
      // stage values stay below 2^14 and, relative to ||a_i||, keep float16's
      // 11 significant bits (entries below 2^-14 are subnormal but then below
      // 2^-6 of the row's largest, with absolute error <= 2^-25).  Any other
      // row is scaled by 2^e_r (largest entry into [1/2, 1)) and stage 3
      // multiplies by 2^-e_r again.  Row r is loaded by the four warps of lane
      // quarter r mod 4, each for a quarter of p.
      __syncthreads();  // every warp is done with the previous tile's row data
      if (tid < TI) rmax[tid] = 0u;
      __syncthreads();
#pragma unroll 1
      for (int rl = 0; rl < 4; ++rl) {
        const int64_t row = i0 + quarter + 4 * rl;
        float mx = 0.f;
        if (row < a.m) {
          const float* arow = a.A + row * a.lda;
          for (int64_t p = 1024 * pq + lane; p < 1024 * pq + 1024 && p < a.n; p += 32)
            mx = fmaxf(mx, fabsf(arow[p]));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) atomicMax(&rmax[quarter + 4 * rl], __float_as_uint(mx));
      }
      __syncthreads();
#pragma unroll 1
      for (int rl = 0; rl < 4; ++rl) {
        const int r = quarter + 4 * rl;
        const int64_t row = i0 + r;
        const bool rv = row < a.m;
        const float* arow = a.A + (rv ? row : 0) * a.lda;
        int ex = 0;
        const float mx = __uint_as_float(rmax[r]);
        if (mx > 0.f) frexpf(mx, &ex);  // mx = f 2^ex, f in [1/2, 1)
        const int e = (mx > 0.f && (ex < -7 || ex > 6)) ? -ex : 0;
        const float sc = ldexpf(1.f, e);
#pragma unroll 1
        for (int p2 = 4 * pq; p2 < 4 * pq + 4; ++p2) {
          uint32_t v[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int p = p2 * 256 + (g + 8 * (j >> 1)) * 16 + 2 * q + 8 * (j & 1);
            const float x0 = (rv && p < a.n) ? arow[p] * sc : 0.f;
            const float x1 = (rv && p + 1 < a.n) ? arow[p + 1] * sc : 0.f;
            v[j] = pack_f16x2(x0, x1);
          }
          tmem_st4(tlane + tcol(rl, p2), v);
        }
        if (pq == 0) {
          // stage-3 A operands W_16 2^-e and 4 I 2^-e, exact in float16 for
          // e in [-13, 24]; the rest of the exponent is undone in float32
          const int ef = e < -13 ? -13 : (e > 24 ? 24 : e);
          const uint32_t mw = f16_pow2(-ef), mi = f16_pow2(2 - ef);
          uint32_t fw[4], fi[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            fw[k] = (aw[k] & 0x80008000u) | mw | (mw << 16);
            fi[k] = ((ai[k] & 0x7fffu) ? mi : 0u) | ((ai[k] & 0x7fff0000u) ? (mi << 16) : 0u);
          }
          rfrag[r * 32 + lane] = make_uint4(fw[0], fw[1], fw[2], fw[3]);
          rfrag[(TI + r) * 32 + lane] = make_uint4(fi[0], fi[1], fi[2], fi[3]);
          if (lane == 0) {
            rrem[r] = e - ef;
            rexp[r] = e;
          }
        }
      }
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      __syncthreads();
      smask = 0u;  // rows of this tile that stage 3 must scale back
#pragma unroll
      for (int r = 0; r < TI; ++r) smask |= rexp[r] != 0 ? (1u << r) : 0u;
      cur_tile = t;
    }

    __syncthreads();  // every warp is done reading E for the previous item

    // Stages 1 and 2 for this warp's rows (quarter + 4 rl) and p2 quarter.
    uint32_t A16[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) A16[e] = ident ? ai[e] : aw[e];
    // 16 units (row slot rl, p2) per warp in p2-major order, two at a time
    // (pair pi: p2 = 4 pq + (pi >> 1), rl = 2 (pi & 1) + h); the next pair's
    // words are loaded from tensor memory while this pair is multiplied.
    auto pair_col = [&](int pi, int h) {
      return tlane + tcol(2 * (pi & 1) + h, 4 * pq + (pi >> 1));
    };
    uint32_t xa[4], xb[4];
    tmem_ld4(pair_col(0, 0), xa);
    tmem_ld4(pair_col(0, 1), xb);
    tmem_wait_ld(xa, xb);
#pragma unroll 1
    for (int pl = 0; pl < 4; ++pl) {
      const int p2 = 4 * pq + pl;
      // float16x2 sign masks of this p2 from its two words (now wd[0], wd[1])
      uint32_t mk[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint32_t t = wd[j >> 1] >> (8 * (j & 1));
        mk[j] = ((t & 1u) << 15) | ((t & 2u) << 30);
      }
#pragma unroll
      for (int hp = 0; hp < 2; ++hp) {
        const int pi = 2 * pl + hp;
        uint32_t x[2][4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          x[0][e] = xa[e] ^ mk[e];
          x[1][e] = xb[e] ^ mk[e];
        }
        if (pi + 1 < 8) {
          tmem_ld4(pair_col(pi + 1, 0), xa);
          tmem_ld4(pair_col(pi + 1, 1), xb);
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int r = quarter + 4 * (2 * hp + h);
          float d1a[4], d1b[4], d2a[4], d2b[4];
          mma16816(d1a, A16, x[h][0], x[h][1]);  // [w0][p1 0..7]
          mma16816(d1b, A16, x[h][2], x[h][3]);  // [w0][p1 8..15]
          mma16816(d2a, A16, pack_f16x2(d1a[0], d1a[1]), pack_f16x2(d1b[0], d1b[1]));  // w0 0..7
          mma16816(d2b, A16, pack_f16x2(d1a[2], d1a[3]), pack_f16x2(d1b[2], d1b[3]));  // w0 8..15
          // [w1][w0] -> E[r][w1][p2][w0 half ^ swizzle]; matrix i = (w1 half i&1, w0 half i>>1)
          const int mi = lane >> 3, mj = lane & 7;
          const int w1 = mj + 8 * (mi & 1), wh = (mi >> 1) ^ ((p2 >> 2) & 1);
          const uint32_t addr = smem_addr(E + r * E_ROW + w1 * E_W1 + p2 * 32 + wh * 16);
          stmatrix_x4(addr, pack_f16x2(d2a[0], d2a[1]), pack_f16x2(d2a[2], d2a[3]),
                      pack_f16x2(d2b[0], d2b[1]), pack_f16x2(d2b[2], d2b[3]));
        }
        tmem_wait_ld(xa, xb);
      }
#pragma unroll
      for (int k = 0; k < 6; ++k) wd[k] = wd[k + 2];
    }
    // the words of the next basis, used by its stages 1-2
    if (item + 1 < ir.end) load_words(b + 1 == int(B) ? 0 : b + 1, wd);
    __syncthreads();  // E holds stages 1-2 of all 16 rows

    // Stage 3: warp handles w1 = warp, 16 rows, one half of w0 at a time.  A
    // tile without scaled rows (the usual case) runs the plain W_16 code.
    auto stage3 = [&](auto scaled_tag) {
    constexpr bool SC = decltype(scaled_tag)::value;
    const int w1 = warp;
#pragma unroll 1
    for (int hh = 0; hh < 2; ++hh) {
      if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
      __syncwarp();  // the previous TMA store has read this warp's F
#pragma unroll 1
      for (int g8 = 0; g8 < 2; ++g8) {
        uint32_t packed[4][4];
#pragma unroll
        for (int rp = 0; rp < 4; ++rp) {
          float v[2][4];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int r = 8 * g8 + 2 * rp + h;
            // lanes 0-15 address p2 = lane & 15 of the w0 half hh (the
            // 16-byte half hh ^ swizzle); the other lanes' addresses are unused
            const int p2 = lane & 15, wh = hh ^ ((p2 >> 2) & 1);
            uint32_t m[2];
            ldmatrix_x2_trans(smem_addr(E + r * E_ROW + w1 * E_W1 + p2 * 32 + wh * 16), m);
            uint32_t A3[4] = {A16[0], A16[1], A16[2], A16[3]};
            bool scaled = false;
            if constexpr (SC) {
              scaled = (smask >> r) & 1u;
              if (scaled) {  // this row's W_16 2^-e_r (or 4 I 2^-e_r)
                const uint4 f4 = rfrag[((ident ? TI : 0) + r) * 32 + lane];
                A3[0] = f4.x;
                A3[1] = f4.y;
                A3[2] = f4.z;
                A3[3] = f4.w;
              }
            }
            mma16816(v[h], A3, m[0], m[1]);  // [w2][w0 8 hh .. 8 hh + 7]
            if (SC && scaled && rrem[r] != 0) {  // beyond float16's exponent range
              const float s3 = ldexpf(1.f, -rrem[r]);
#pragma unroll
              for (int e = 0; e < 4; ++e) v[h][e] *= s3;
            }
          }
#pragma unroll
          for (int pos = 0; pos < 4; ++pos) packed[pos][rp] = pack_bf16x2(v[0][pos], v[1][pos]);
        }
        // position pos: w2 = g + 8 (pos >> 1), w0 = 8 hh + 2q + (pos & 1).
        // F is [w2][w0 - 8 hh][row] under the tensor map's 32-byte swizzle:
        // the 16-byte half g8 of the 32-byte row (w2, w0') sits at g8 ^ (bit 2
        // of w0').  Lanes of odd g store the positions of a pair in the other
        // order, so the eight lanes of a quarter-warp cover all eight bank
        // slots: (bit 0 of w0') ^ (g & 1), bit 1 of w0', half.
        const bool swp = g & 1;
#pragma unroll
        for (int pos = 0; pos < 4; ++pos) {
          const int ps = swp ? pos ^ 1 : pos;
          const int w2 = g + 8 * (pos >> 1), w0 = 2 * q + (ps & 1);
          const int half = g8 ^ ((w0 >> 2) & 1);
          uint4 val;
          val.x = swp ? packed[pos ^ 1][0] : packed[pos][0];
          val.y = swp ? packed[pos ^ 1][1] : packed[pos][1];
          val.z = swp ? packed[pos ^ 1][2] : packed[pos][2];
          val.w = swp ? packed[pos ^ 1][3] : packed[pos][3];
          *reinterpret_cast<uint4*>(Fw + (w2 * 8 + w0) * (TI * 2) + half * 16) = val;
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0 && aligned) {
        tma_store_4d(&tmap, smem_addr(Fw), int(i0), 8 * hh, w1, b * 16);
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      }
    }
    };
    if (smask == 0u)
      stage3(std::integral_constant<bool, false>{});
    else
      stage3(std::integral_constant<bool, true>{});
  }
  if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encoder() {
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

}  // namespace tc

int launch_d4096_tc(const Plan& p) {
  tc::EncodeTiledFn enc = tc::encoder();
  if (enc == nullptr) return KERDOCK_ERR_UNSUPPORTED;
  // R[b][w][i] (bfloat16) as [(b, w2)][w1][w0][i]: box 16 rows x 8 w0 x 1 w1 x 16 w2
  CUtensorMap map;
  const cuuint64_t dims[4] = {cuuint64_t(p.ldr), 16, 16, cuuint64_t(p.B) * 16};
  const cuuint64_t strides[3] = {cuuint64_t(p.ldr) * 2, cuuint64_t(p.ldr) * 32,
                                 cuuint64_t(p.ldr) * 512};
  const cuuint32_t box[4] = {tc::TI, 8, 1, 16};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, p.repr, dims, strides, box, es,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
          CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return KERDOCK_ERR_UNSUPPORTED;
  auto kern = tc::preprocess_d4096_tc_kernel;
  KD_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   int(tc::SMEM)));
  PreArgs a;
  a.A = p.A;
  a.lda = p.lda;
  a.m = p.m;
  a.n = p.n;
  a.signs = p.signs();
  a.sign_words = p.sign_words;
  a.R = p.repr;
  a.ldr = p.ldr;
  a.status = p.status();
  a.num_tiles = (p.ldr + tc::TI - 1) / tc::TI;
  // groups of up to 8 CTAs (one per SM) on adjacent 16-row tiles: 152 SMs
  // are 19 such groups (groups of 16 would leave 8 SMs idle; a store-only
  // probe of the pattern runs as fast with groups of 4 as of 16)
  a.group = pick_group(a.num_tiles, 8);
  int64_t ngrp = int64_t(p.num_sms) / a.group;
  const int64_t items = ((a.num_tiles + a.group - 1) / a.group) * p.B;
  if (ngrp > items) ngrp = items;
  if (ngrp < 1) ngrp = 1;
  kern<<<unsigned(ngrp * a.group), tc::THREADS, tc::SMEM, p.stream>>>(a, map);
  KD_CUDA_TRY(cudaGetLastError());
  return KERDOCK_OK;
}

// ---------------------------------------------------------------------------
// d = 4096, float32 representation, on the tensor cores
// (preprocess_d4096_tc32_kernel).  The three stages of
// preprocess_d4096_tc_kernel with float32 accuracy: every float16 data operand
// is a pair hi + lo (hi = float16(v), lo = float16(v - hi): 22 significant
// bits together), and W_16, exact in float16, multiplies both into one
// float32 accumulator (two MMAs per product).  Every row is scaled by 2^e_r
// (largest entry into [1/2, 1)) before the split, so the pair keeps 22 bits of
// each entry down to 2^-3 of the row's largest and an absolute 2^-25 below
// that (lo becomes subnormal); stage 3 multiplies by 2^-e_r in float32.  A
// CTA's tile is 8 rows (32-byte float32 runs, as 16 rows of bfloat16), E
// holds the hi and lo planes of stages 1-2 and tensor memory the hi and lo
// words of the tile, so both take the bfloat16 kernel's space and each item
// the same number of MMAs for the same 128 KiB of output.
// ---------------------------------------------------------------------------
namespace tc32 {

using tc::ldmatrix_x2_trans;
using tc::mma16816;
using tc::pack_f16x2;
using tc::stmatrix_x4;
using tc::tma_store_4d;

constexpr int TI = 8, WARPS = 16, THREADS = WARPS * 32, D = 4096;
constexpr int E_W1 = 16 * 32 + 16;      // bytes per (row, w1) of one plane: 16 p2 x 32 B + pad
constexpr int E_ROW = 16 * E_W1;        // bytes per row of one plane
constexpr int E_PLANE = TI * E_ROW;     // 67584: hi plane, then lo plane
constexpr int E_BYTES = 2 * E_PLANE;
constexpr int F_WARP = 16 * 8 * TI * 4;  // [w2][w0 half][row] float32 per warp: 4 KiB
constexpr size_t OFF_SLOT = size_t(E_BYTES) + size_t(WARPS) * F_WARP;
constexpr size_t OFF_RMAX = OFF_SLOT + 16;
constexpr size_t OFF_RSC = OFF_RMAX + TI * 4;
constexpr size_t SMEM = OFF_RSC + TI * 4;
constexpr uint32_t TMEM_COLS = 256;  // 2 rows x 16 p2 x (4 hi + 4 lo) words per lane

// Column of tensor memory holding a thread's eight words (hi 0-3, lo 4-7) for (row slot rl, p2).
__device__ __forceinline__ uint32_t tcol(int rl, int p2) { return uint32_t((rl * 16 + p2) * 8); }

// d += A B (float32 accumulator in and out)
__device__ __forceinline__ void mma16816_acc(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                             uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
// (v0, v1) as float16x2 pairs hi + lo
__device__ __forceinline__ void split2(float v0, float v1, uint32_t& hi, uint32_t& lo) {
  const __half2 h = __floats2half2_rn(v0, v1);
  const float2 hf = __half22float2(h);
  const __half2 l = __floats2half2_rn(v0 - hf.x, v1 - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&v)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                 "=r"(v[6]), "=r"(v[7])
               : "r"(taddr)
               : "memory");
}
// Loads are asynchronous: the registers are valid after this wait, which
// names them so that the compiler does not read them earlier.
__device__ __forceinline__ void tmem_wait_ld8(uint32_t (&u)[8], uint32_t (&v)[8]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(u[0]), "+r"(u[1]), "+r"(u[2]), "+r"(u[3]), "+r"(u[4]), "+r"(u[5]),
                 "+r"(u[6]), "+r"(u[7]), "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]),
                 "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7])
               :
               : "memory");
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&v)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(
                   taddr),
               "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]),
               "r"(v[7])
               : "memory");
}

__global__ void __launch_bounds__(THREADS, 1)
    preprocess_d4096_tc32_kernel(const PreArgs a, const __grid_constant__ CUtensorMap tmap) {
  constexpr int64_t B = D / 2 + 1;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* E = smem;
  unsigned char* Fw = smem + E_BYTES + (threadIdx.x >> 5) * F_WARP;  // this warp's F
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + OFF_SLOT);
  uint32_t* rmax = reinterpret_cast<uint32_t*>(smem + OFF_RMAX);  // row maxima (float bits)
  float* rsc = reinterpret_cast<float*>(smem + OFF_RSC);          // 2^-e_r
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, q = lane & 3;
  const int quarter = warp & 3, pq = warp >> 2;  // lane quarter of tensor memory; p2 quarter
  const bool aligned = (smem_addr(smem) & 1023u) == 0;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(tmem_slot);
  const uint32_t tlane = tmem + (uint32_t(quarter * 32) << 16);
  if (tid == 0 && !aligned) set_status(a.status, kStatusBadIndex);

  // A fragments (rows g, g+8; columns 2q, 2q+1, 2q+8, 2q+9) of W_16 and of 4 I.
  uint32_t aw[4], ai[4];
  {
    const int rr[4] = {g, g + 8, g, g + 8};
    const int cc[4] = {2 * q, 2 * q, 2 * q + 8, 2 * q + 8};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float w0 = (__popc(rr[e] & cc[e]) & 1) ? -1.f : 1.f;
      const float w1 = (__popc(rr[e] & (cc[e] + 1)) & 1) ? -1.f : 1.f;
      aw[e] = pack_f16x2(w0, w1);
      ai[e] = pack_f16x2(rr[e] == cc[e] ? 4.f : 0.f, rr[e] == cc[e] + 1 ? 4.f : 0.f);
    }
  }

  const ItemRange ir = item_range(blockIdx.x, gridDim.x, a.group, a.num_tiles, B);
  // Step (i) of Lemma 6 in registers, as in preprocess_d4096_tc_kernel: the
  // warp's p2 quarter needs two sign words per p2, requested for the next
  // basis while stage 3 of this one runs.
  const int wsh = 16 * (g & 1) + 2 * q;
  auto load_words = [&](int b, uint32_t (&wd)[8]) {
    const uint32_t* srow =
        a.signs + int64_t(b == D / 2 ? 0 : b) * a.sign_words + 32 * pq + (g >> 1);
#pragma unroll
    for (int k = 0; k < 8; ++k)
      wd[k] = b == D / 2 ? 0u : __ldg(srow + 8 * (k >> 1) + 4 * (k & 1)) >> wsh;
  };
  uint32_t wd[8];
  if (ir.beg < ir.end) load_words(int(ir.beg % B), wd);
  int64_t cur_tile = -1;
  for (int64_t item = ir.beg; item < ir.end; ++item) {
    const int64_t tg = item / B;
    const int b = int(item - tg * B);
    const int64_t t = tg * a.group + ir.slot;
    const int64_t i0 = t * TI;
    const bool ident = b == D / 2;

    if (t != cur_tile) {  // this warp's share of the tile into its lanes of tensor memory
      // Row r is loaded by the four warps of lane quarter r mod 4, each for a
      // quarter of p, scaled by 2^e_r (|e_r| <= 126) and split into hi + lo.
      __syncthreads();  // every warp is done with the previous tile's row data
      if (tid < TI) rmax[tid] = 0u;
      __syncthreads();
#pragma unroll 1
      for (int rl = 0; rl < 2; ++rl) {
        const int64_t row = i0 + quarter + 4 * rl;
        float mx = 0.f;
        if (row < a.m) {
          const float* arow = a.A + row * a.lda;
          for (int64_t p = 1024 * pq + lane; p < 1024 * pq + 1024 && p < a.n; p += 32)
            mx = fmaxf(mx, fabsf(arow[p]));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) atomicMax(&rmax[quarter + 4 * rl], __float_as_uint(mx));
      }
      __syncthreads();
#pragma unroll 1
      for (int rl = 0; rl < 2; ++rl) {
        const int r = quarter + 4 * rl;
        const int64_t row = i0 + r;
        const bool rv = row < a.m;
        const float* arow = a.A + (rv ? row : 0) * a.lda;
        int ex = 0;
        const float mx = __uint_as_float(rmax[r]);
        if (mx > 0.f) frexpf(mx, &ex);  // mx = f 2^ex, f in [1/2, 1)
        int e = mx > 0.f ? -ex : 0;
        e = e > 126 ? 126 : (e < -126 ? -126 : e);
        const float sc = ldexpf(1.f, e);
        if (pq == 0 && lane == 0) rsc[r] = ldexpf(1.f, -e);
#pragma unroll 1
        for (int p2 = 4 * pq; p2 < 4 * pq + 4; ++p2) {
          uint32_t v[8];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int p = p2 * 256 + (g + 8 * (j >> 1)) * 16 + 2 * q + 8 * (j & 1);
            const float x0 = (rv && p < a.n) ? arow[p] * sc : 0.f;
            const float x1 = (rv && p + 1 < a.n) ? arow[p + 1] * sc : 0.f;
            split2(x0, x1, v[j], v[4 + j]);
          }
          tmem_st8(tlane + tcol(rl, p2), v);
        }
      }
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      cur_tile = t;
    }

    __syncthreads();  // every warp is done reading E for the previous item

    // Stages 1 and 2 for this warp's rows (quarter, quarter + 4) and p2
    // quarter: for each p2 the two rows, with the next p2's words loaded from
    // tensor memory while these are multiplied.
    uint32_t A16[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) A16[e] = ident ? ai[e] : aw[e];
    uint32_t xa[8], xb[8];
    tmem_ld8(tlane + tcol(0, 4 * pq), xa);
    tmem_ld8(tlane + tcol(1, 4 * pq), xb);
    tmem_wait_ld8(xa, xb);
#pragma unroll 1
    for (int pl = 0; pl < 4; ++pl) {
      const int p2 = 4 * pq + pl;
      // float16x2 sign masks of this p2 from its two words (now wd[0], wd[1]);
      // they flip hi and lo alike
      uint32_t mk[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint32_t u = wd[j >> 1] >> (8 * (j & 1));
        mk[j] = ((u & 1u) << 15) | ((u & 2u) << 30);
      }
      uint32_t x[2][8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        x[0][e] = xa[e] ^ mk[e & 3];
        x[1][e] = xb[e] ^ mk[e & 3];
      }
      if (pl < 3) {
        tmem_ld8(tlane + tcol(0, p2 + 1), xa);
        tmem_ld8(tlane + tcol(1, p2 + 1), xb);
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = quarter + 4 * h;
        float d1a[4], d1b[4];
        mma16816(d1a, A16, x[h][0], x[h][1]);  // [w0][p1 0..7]
        mma16816_acc(d1a, A16, x[h][4], x[h][5]);
        mma16816(d1b, A16, x[h][2], x[h][3]);  // [w0][p1 8..15]
        mma16816_acc(d1b, A16, x[h][6], x[h][7]);
        uint32_t bh[4], bl[4];
        split2(d1a[0], d1a[1], bh[0], bl[0]);
        split2(d1b[0], d1b[1], bh[1], bl[1]);
        split2(d1a[2], d1a[3], bh[2], bl[2]);
        split2(d1b[2], d1b[3], bh[3], bl[3]);
        float d2a[4], d2b[4];
        mma16816(d2a, A16, bh[0], bh[1]);  // w0 0..7
        mma16816_acc(d2a, A16, bl[0], bl[1]);
        mma16816(d2b, A16, bh[2], bh[3]);  // w0 8..15
        mma16816_acc(d2b, A16, bl[2], bl[3]);
        uint32_t eh[4], el[4];
        split2(d2a[0], d2a[1], eh[0], el[0]);
        split2(d2a[2], d2a[3], eh[1], el[1]);
        split2(d2b[0], d2b[1], eh[2], el[2]);
        split2(d2b[2], d2b[3], eh[3], el[3]);
        // [w1][w0] -> E[plane][r][w1][p2][w0 half ^ swizzle]; matrix i = (w1 half i&1, w0 half i>>1)
        const int mi = lane >> 3, mj = lane & 7;
        const int w1 = mj + 8 * (mi & 1), wh = (mi >> 1) ^ ((p2 >> 2) & 1);
        const uint32_t addr = smem_addr(E + r * E_ROW + w1 * E_W1 + p2 * 32 + wh * 16);
        stmatrix_x4(addr, eh[0], eh[1], eh[2], eh[3]);
        stmatrix_x4(addr + E_PLANE, el[0], el[1], el[2], el[3]);
      }
      if (pl < 3) tmem_wait_ld8(xa, xb);
#pragma unroll
      for (int k = 0; k < 6; ++k) wd[k] = wd[k + 2];
    }
    // the words of the next basis, used by its stages 1-2
    if (item + 1 < ir.end) load_words(b + 1 == int(B) ? 0 : b + 1, wd);
    __syncthreads();  // E holds stages 1-2 of all 8 rows

    // Stage 3: warp handles w1 = warp, 8 rows, one half of w0 at a time.
    const int w1 = warp;
    const bool swp = g & 1;
#pragma unroll 1
    for (int hh = 0; hh < 2; ++hh) {
      float v[TI][4];
#pragma unroll
      for (int r = 0; r < TI; ++r) {
        // lanes 0-15 address p2 = lane & 15 of the w0 half hh (the 16-byte
        // half hh ^ swizzle); the other lanes' addresses are unused
        const int p2 = lane & 15, wh = hh ^ ((p2 >> 2) & 1);
        const uint32_t addr = smem_addr(E + r * E_ROW + w1 * E_W1 + p2 * 32 + wh * 16);
        uint32_t mh[2], ml[2];
        ldmatrix_x2_trans(addr, mh);
        ldmatrix_x2_trans(addr + E_PLANE, ml);
        mma16816(v[r], A16, mh[0], mh[1]);  // [w2][w0 8 hh .. 8 hh + 7]
        mma16816_acc(v[r], A16, ml[0], ml[1]);
        const float s = rsc[r];
#pragma unroll
        for (int e = 0; e < 4; ++e) v[r][e] *= s;
      }
      if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
      __syncwarp();  // the previous TMA store has read this warp's F
      // position pos: w2 = g + 8 (pos >> 1), w0 = 8 hh + 2q + (pos & 1).  F is
      // [w2][w0 - 8 hh][row] (32-byte rows) under the tensor map's 32-byte
      // swizzle: rows 4 r4 .. 4 r4 + 3 of (w2, w0') sit in the 16-byte half
      // r4 ^ (bit 2 of w0').  Odd-g lanes store the positions of a pair in the
      // other order, so a quarter-warp covers all eight bank slots.
#pragma unroll
      for (int r4 = 0; r4 < 2; ++r4) {
#pragma unroll
        for (int pos = 0; pos < 4; ++pos) {
          const int ps = swp ? pos ^ 1 : pos;
          const int w2 = g + 8 * (pos >> 1), w0 = 2 * q + (ps & 1);
          const int half = r4 ^ ((w0 >> 2) & 1);
          uint4 val;
          val.x = __float_as_uint(swp ? v[4 * r4][pos ^ 1] : v[4 * r4][pos]);
          val.y = __float_as_uint(swp ? v[4 * r4 + 1][pos ^ 1] : v[4 * r4 + 1][pos]);
          val.z = __float_as_uint(swp ? v[4 * r4 + 2][pos ^ 1] : v[4 * r4 + 2][pos]);
          val.w = __float_as_uint(swp ? v[4 * r4 + 3][pos ^ 1] : v[4 * r4 + 3][pos]);
          *reinterpret_cast<uint4*>(Fw + (w2 * 8 + w0) * (TI * 4) + half * 16) = val;
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0 && aligned) {
        tma_store_4d(&tmap, smem_addr(Fw), int(i0), 8 * hh, w1, b * 16);
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      }
    }
  }
  if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
}

}  // namespace tc32

int launch_d4096_tc32(const Plan& p) {
  tc::EncodeTiledFn enc = tc::encoder();
  if (enc == nullptr) return KERDOCK_ERR_UNSUPPORTED;
  // R[b][w][i] (float32) as [(b, w2)][w1][w0][i]: box 8 rows x 8 w0 x 1 w1 x 16 w2
  CUtensorMap map;
  const cuuint64_t dims[4] = {cuuint64_t(p.ldr), 16, 16, cuuint64_t(p.B) * 16};
  const cuuint64_t strides[3] = {cuuint64_t(p.ldr) * 4, cuuint64_t(p.ldr) * 64,
                                 cuuint64_t(p.ldr) * 1024};
  const cuuint32_t box[4] = {tc32::TI, 8, 1, 16};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, p.repr, dims, strides, box, es,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
          CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return KERDOCK_ERR_UNSUPPORTED;
  auto kern = tc32::preprocess_d4096_tc32_kernel;
  KD_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   int(tc32::SMEM)));
  PreArgs a;
  a.A = p.A;
  a.lda = p.lda;
  a.m = p.m;
  a.n = p.n;
  a.signs = p.signs();
  a.sign_words = p.sign_words;
  a.R = p.repr;
  a.ldr = p.ldr;
  a.status = p.status();
  a.num_tiles = (p.ldr + tc32::TI - 1) / tc32::TI;
  // groups of up to 8 CTAs (one per SM) on adjacent 8-row tiles, as for the
  // bfloat16 kernel
  a.group = pick_group(a.num_tiles, 8);
  int64_t ngrp = int64_t(p.num_sms) / a.group;
  const int64_t items = ((a.num_tiles + a.group - 1) / a.group) * p.B;
  if (ngrp > items) ngrp = items;
  if (ngrp < 1) ngrp = 1;
  kern<<<unsigned(ngrp * a.group), tc32::THREADS, tc32::SMEM, p.stream>>>(a, map);
  KD_CUDA_TRY(cudaGetLastError());
  return KERDOCK_OK;
}

// ---------------------------------------------------------------------------
// d = 1024, float32 or bfloat16 representation.  Write p = 32 s + k and
// w = 32 w_hi + w_lo, so W_1024 = W_32 (over s) (x) W_32 (over k).  The CTA's
// 16-row tile of A lives in tensor memory: thread (row pair rp, source s)
// keeps rows 2 rp and 2 rp + 1 at p in [32 s, 32 s + 32) as 64 words of its
// own lane, so shared memory holds only the exchange buffer.  Per basis:
// phase 1 reads the 64 words back (tcgen05.ld), flips both rows of a p with
// the same sign bit (step (i) of Lemma 6; the two rows share the sign word)
// and runs the five stages over k packed across the row pair; one exchange
// of 8-byte row pairs X[s][w_lo][row] (conflict-free); phase 2, thread
// (rp, w_lo), runs the five stages over s and stores 16 x 2-row runs as the
// other kernels do.  Two barriers per basis, and a thread's phase 1 of the
// next basis overlaps the other warps' phase 2.
namespace k10 {

constexpr int D = 1024, NS = 32;

// TI-row tiles: TI / 2 row pairs x 32 sources = one thread each.
template <int TI>
struct Cfg {
  static constexpr int RP = TI / 2;
  static constexpr int THREADS = RP * NS;
  static constexpr int XST = 32 * TI + 16;  // floats per source: [w_lo][row] + 16 (bank shift)
  static constexpr size_t SMEM = size_t(NS) * XST * 4 + 16;
  static constexpr uint32_t TMEM_COLS = uint32_t(THREADS) * 64 / 128;  // 64 words per thread
};

// Asynchronous: the registers are valid after tmem_wait16 has named them.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15])
      : "r"(taddr)
      : "memory");
}
// One wait for all loads issued so far; each group of 16 registers is then
// named so that no read of them moves above the wait.
__device__ __forceinline__ void tmem_wait64(uint32_t (&v)[64]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 64; i += 16)
    asm volatile(""
                 : "+r"(v[i + 0]), "+r"(v[i + 1]), "+r"(v[i + 2]), "+r"(v[i + 3]), "+r"(v[i + 4]),
                   "+r"(v[i + 5]), "+r"(v[i + 6]), "+r"(v[i + 7]), "+r"(v[i + 8]), "+r"(v[i + 9]),
                   "+r"(v[i + 10]), "+r"(v[i + 11]), "+r"(v[i + 12]), "+r"(v[i + 13]),
                   "+r"(v[i + 14]), "+r"(v[i + 15]));
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
      "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]),
      "r"(v[15])
      : "memory");
}

template <typename OutT, int TI>
__global__ void __launch_bounds__(Cfg<TI>::THREADS, TI == 16 ? 2 : 1)
    preprocess_d1024_kernel(const PreArgs a) {
  using C = Cfg<TI>;
  constexpr int XST = C::XST, RP = C::RP;
  constexpr uint32_t TMEM_COLS = C::TMEM_COLS;
  constexpr int64_t B = D / 2 + 1;
  extern __shared__ __align__(16) float smem[];
  float* X = smem;  // [NS][XST]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + NS * XST);
  OutT* R = static_cast<OutT*>(a.R);
  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int rp = lane % RP;                       // rows 2 rp, 2 rp + 1 (both phases)
  const int s = lane / RP + (32 / RP) * g;        // phase 1: source s; phase 2: w_lo = s
  const float sqrt_d = 32.f;

  if (g == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(tmem_slot);
  // warp g reaches lanes 32 (g mod 4) ..; warps 4 j .. 4 j + 3 use columns 64 j ..
  const uint32_t tme = tmem + (uint32_t((g & 3) * 32) << 16) + uint32_t((g >> 2) * 64);

  const ItemRange ir = item_range(blockIdx.x, gridDim.x, a.group, a.num_tiles, B);
  // sign word of basis b for this thread's p range (zero for the identity basis)
  auto sign_word = [&](int b) {
    return b == D / 2 ? 0u : __ldg(a.signs + int64_t(b) * a.sign_words + s);
  };
  uint32_t sw_next = ir.beg < ir.end ? sign_word(int(ir.beg % B)) : 0u;
  int64_t cur_tile = -1;
  for (int64_t item = ir.beg; item < ir.end; ++item) {
    const int64_t tg = item / B;
    const int b = int(item - tg * B);
    const int64_t t = tg * a.group + ir.slot;
    const int64_t i0 = t * TI;
    const bool ident = b == D / 2;
    if (t != cur_tile) {  // this thread's 64 words: (row 2 rp, row 2 rp + 1) per p
#pragma unroll 1
      for (int c = 0; c < 4; ++c) {
        uint32_t w[16];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int p = 32 * s + 8 * c + e;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int64_t row = i0 + 2 * rp + h;
            const float v = (row < a.m && p < a.n) ? a.A[row * a.lda + p] : 0.f;
            w[2 * e + h] = __float_as_uint(v);
          }
        }
        tmem_st16(tme + uint32_t(16 * c), w);
      }
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      cur_tile = t;
    }
    // Phase 1: k in registers, (row 2 rp, row 2 rp + 1) packed; the four
    // tensor-memory loads and the sign word are in flight together.
    uint32_t w[64];
#pragma unroll
    for (int c = 0; c < 4; ++c) tmem_ld16(tme + uint32_t(16 * c), w + 16 * c);
    // this basis's sign word was requested one basis ahead; request the next
    const uint32_t sw = sw_next;
    if (item + 1 < ir.end) sw_next = sign_word(b + 1 == int(B) ? 0 : b + 1);
    tmem_wait64(w);
    float2 v[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      const uint32_t f = (sw << (31 - k)) & 0x80000000u;
      v[k] = make_float2(__uint_as_float(w[2 * k] ^ f), __uint_as_float(w[2 * k + 1] ^ f));
    }
    if (!ident) fwht_across<32>(v);
    __syncthreads();  // every warp is done reading X for the previous basis
#pragma unroll
    for (int k = 0; k < 32; ++k) *reinterpret_cast<float2*>(&X[s * XST + k * TI + 2 * rp]) = v[k];
    __syncthreads();

    // Phase 2: thread (rp, w_lo = s) combines the 32 sources.
    float2 y[32];
#pragma unroll
    for (int h = 0; h < 32; ++h) y[h] = *reinterpret_cast<const float2*>(&X[h * XST + s * TI + 2 * rp]);
    if (!ident) {
      fwht_across<32>(y);
    } else {
#pragma unroll
      for (int h = 0; h < 32; ++h) y[h] = make_float2(y[h].x * sqrt_d, y[h].y * sqrt_d);
    }
    const int64_t orow = i0 + 2 * rp;
    if (orow < a.ldr) {
      OutT* rb = R + (int64_t(b) * D + s) * a.ldr + orow;  // w = 32 h + s
#pragma unroll
      for (int h = 0; h < 32; ++h) store_pair<OutT>(rb + int64_t(h) * 32 * a.ldr, y[h]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (g == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
}

}  // namespace k10

template <typename OutT>
int launch_d1024(const Plan& p) {
  // 16-row tiles, two CTAs per SM.  32-row tiles (one CTA of 16 warps per SM,
  // twice the run length per output row) measured slower for both types:
  // 0.495 vs 0.437 ms (float32) and 0.435 vs 0.420 ms (bfloat16), the SM
  // idling at the CTA's two barriers per basis.
  constexpr int TI = 16;
  using C = k10::Cfg<TI>;
  auto kern = k10::preprocess_d1024_kernel<OutT, TI>;
  KD_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   int(C::SMEM)));
  // the whole unified L1 as shared memory
  KD_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                   int(cudaSharedmemCarveoutMaxShared)));
  // CTAs per SM from the kernel's registers and shared memory (the runtime's
  // occupancy query reported one for the 16-row kernel, though two fit), and at
  // most what the SM's 512 tensor-memory columns hold
  cudaFuncAttributes fa;
  KD_CUDA_TRY(cudaFuncGetAttributes(&fa, kern));
  int dev = 0, regs_sm = 0, smem_sm = 0, smem_rsv = 0;
  KD_CUDA_TRY(cudaGetDevice(&dev));
  KD_CUDA_TRY(cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev));
  KD_CUDA_TRY(
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
  KD_CUDA_TRY(cudaDeviceGetAttribute(&smem_rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev));
  const int regs_cta = ((fa.numRegs + 7) / 8 * 8) * C::THREADS;  // 8-register granules
  int occ = regs_cta > 0 ? regs_sm / regs_cta : 1;
  const int by_smem = smem_sm / int(C::SMEM + size_t(fa.sharedSizeBytes) + size_t(smem_rsv));
  if (by_smem < occ) occ = by_smem;
  if (occ > int(512 / C::TMEM_COLS)) occ = int(512 / C::TMEM_COLS);  // 512 columns per SM
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
  a.status = p.status();
  a.num_tiles = (p.ldr + TI - 1) / TI;
  // groups of CTAs on adjacent tiles covering 256 consecutive rows
  a.group = pick_group(a.num_tiles, 256 / TI);
  int64_t ngrp = int64_t(p.num_sms) * occ / a.group;
  const int64_t items = ((a.num_tiles + a.group - 1) / a.group) * p.B;
  if (ngrp > items) ngrp = items;
  if (ngrp < 1) ngrp = 1;
  kern<<<unsigned(ngrp * a.group), C::THREADS, C::SMEM, p.stream>>>(a);
  KD_CUDA_TRY(cudaGetLastError());
  return KERDOCK_OK;
}

// ---------------------------------------------------------------------------
// d = 1024, bfloat16 representation on the tensor cores.  Write
// p = 256 p2 + 16 p1 + p0 and w = 256 w2 + 16 w1 + w0, so that
// W_1024 = W_4 (over p2) (x) W_16 (over p1) (x) W_16 (over p0).  A CTA owns a
// 64-row tile of A, kept in tensor memory as float16 (each row scaled by a
// power of two into [1/2, 1)) across all the bases it processes.  Per basis
// each warp takes 8 rows: step (i) of Lemma 6 is an XOR of the float16 sign
// bits, the 4-point stage over p2 runs on the input in packed float16 and goes
// back to tensor memory.  Then, for each output quarter w2, two mma.sync
// stages (float16 operands, float32 accumulation) over p0 and p1 -- the first
// stage's accumulators are exactly the second stage's B fragments -- give the
// quarter's 256 outputs of a row; the row's power-of-two scale is undone in
// the second stage's A operand.  Eight rows are packed per 16-byte store into
// a staging buffer [w][64 rows] (128-byte swizzle), and one TMA store writes
// 64 rows x 256 w, i.e. 128-byte runs of every output row R[b][w][.].
// Float16 keeps 11 significant bits, so the stages add only a few 2^-11
// ||a_i|| to the final bfloat16 rounding (2^-9 |R|).
// ---------------------------------------------------------------------------
namespace k10tc {

constexpr int D = 1024, TI = 64, WARPS = 8, THREADS = WARPS * 32, RPW = TI / WARPS;
constexpr int QW = 256;                         // outputs w per quarter
static_assert(THREADS == QW, "the identity basis gives each thread one w of a quarter");
constexpr int FBUF = QW * TI * 2;               // 32 KiB: one quarter's staging
constexpr int NBUF = 4;                         // two rounds of two quarters
constexpr int MASKW = 512;                      // float16 sign masks per basis (16 per lane)
constexpr size_t OFF_MASK = size_t(NBUF) * FBUF;
constexpr size_t OFF_FRAG = OFF_MASK + 2 * MASKW * 4;                    // [warp][row][lane] uint4
constexpr size_t OFF_ER = OFF_FRAG + size_t(WARPS) * RPW * 32 * 16;     // [warp][row] int
constexpr size_t OFF_SLOT = OFF_ER + size_t(WARPS) * RPW * 4;
constexpr size_t OFF_SCR = OFF_SLOT + 16;                               // [warp][512] half2 words
constexpr size_t SMEM = OFF_SCR + size_t(WARPS) * 512 * 4 + 1024;  // + slack for 1024-byte alignment
constexpr uint32_t TMEM_COLS = 512;             // per warp: 128 columns of x, 128 of y

__device__ __forceinline__ uint32_t pack_h2(float lo, float hi) {
  const __half2 h = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&h);
}
__device__ __forceinline__ uint32_t pack_b2(float lo, float hi) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&h);
}
__device__ __forceinline__ uint32_t hadd2(uint32_t a, uint32_t b) {
  uint32_t r;
  asm("add.rn.f16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}
__device__ __forceinline__ uint32_t hsub2(uint32_t a, uint32_t b) {
  uint32_t r;
  asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}
__device__ __forceinline__ void mma_f16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                        uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%10,%10,%10,%10};"
      : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1), "f"(0.f));
}
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t (&v)[4]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
               : "r"(taddr)
               : "memory");
}
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, uint32_t src, int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
          reinterpret_cast<uint64_t>(map)),
      "r"(c0), "r"(c1), "r"(src)
      : "memory");
}

__global__ void __launch_bounds__(THREADS, 1)
    preprocess_d1024_tc_kernel(const PreArgs a, const __grid_constant__ CUtensorMap tmap) {
  constexpr int64_t B = D / 2 + 1;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
  uint32_t* masks = reinterpret_cast<uint32_t*>(smem + OFF_MASK);  // [2][4][32 lanes][4]
  uint4* frag = reinterpret_cast<uint4*>(smem + OFF_FRAG);         // [warp][row][lane]
  int* erem = reinterpret_cast<int*>(smem + OFF_ER);                // [warp][row]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + OFF_SLOT);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, q = lane & 3;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(tmem_slot);
  // warp w reaches lanes 32 (w mod 4) ..; warps 4 .. 7 use columns 256 ..
  const uint32_t tx = tmem + (uint32_t((warp & 3) * 32) << 16) + uint32_t((warp >> 2) * 256);
  const uint32_t ty = tx + 128;

  // A fragment of W_16 in float16 (rows g, g + 8; columns 2q, 2q + 1, 2q + 8, 2q + 9)
  uint32_t w16[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int r = g + 8 * (e & 1), c = 2 * q + 8 * (e >> 1);
    const uint32_t lo = (__popc(r & c) & 1) ? 0xBC00u : 0x3C00u;
    const uint32_t hi = (__popc(r & (c + 1)) & 1) ? 0xBC00u : 0x3C00u;
    w16[e] = lo | (hi << 16);
  }

  // Float16 sign masks of basis b in the lanes' fragment order: mask word
  // (lane, reg) flips the elements p and p + 1 of B-fragment register reg =
  // 4 p2 + 2 nt + j, p = 256 p2 + 16 (g + 8 nt) + 2 q + 8 j.
  // Thread tid builds the masks idx = tid and tid + THREADS; the sign words
  // are requested early (sign_words) and turned into masks later (put_masks).
  static_assert(MASKW == 2 * THREADS, "two mask words per thread");
  auto mask_p = [](int idx) {
    const int l = idx >> 4, reg = idx & 15;
    return 256 * (reg >> 2) + 16 * ((l >> 2) + 8 * ((reg >> 1) & 1)) + 2 * (l & 3) +
           8 * (reg & 1);
  };
  auto sign_words = [&](int b, uint32_t (&wd)[2]) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int p = mask_p(tid + h * THREADS);
      wd[h] = b != D / 2 ? __ldg(a.signs + int64_t(b) * a.sign_words + (p >> 5)) : 0u;
    }
  };
  auto put_masks = [&](const uint32_t (&wd)[2], int mb) {
    uint32_t* mk = masks + mb * MASKW;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int idx = tid + h * THREADS, l = idx >> 4, reg = idx & 15;
      const uint32_t bits = wd[h] >> (mask_p(idx) & 31);
      mk[((reg >> 2) * 32 + l) * 4 + (reg & 3)] = ((bits & 1u) << 15) | ((bits & 2u) << 30);
    }
  };
  auto build_masks = [&](int b, int mb) {
    uint32_t wd[2];
    sign_words(b, wd);
    put_masks(wd, mb);
  };
  uint32_t wd_next[2] = {0u, 0u};  // sign words of the grab's next basis, requested early

  // Dynamic schedule: CTA c starts on tile c mod T and takes CH bases at a
  // time from that tile's counter; when its tile has none left it moves to
  // the next tile that has (a tile reload), so SMs that write more slowly
  // than others do not set the kernel's time.
  // The last item of a grab already takes the next one (thread 0, during its
  // first phase, into the other slot of s_grab), so the next grab's first
  // masks are prepared like any other basis's.
  __shared__ int s_grab[2][2];  // [slot][tile, first basis (-1: none left)]
  constexpr int CH = 8;
  const int T = int(a.num_tiles);
  auto grab = [&](int from, int slot) {  // thread 0 only
    int gt = -1, gb = -1;
    for (int k = 0; k < T && gb < 0; ++k) {
      const int tt = (from + k) % T;
      if (*reinterpret_cast<volatile int*>(a.work + tt) >= int(B)) continue;
      const int got = atomicAdd(a.work + tt, CH);
      if (got < int(B)) {
        gt = tt;
        gb = got;
      }
    }
    s_grab[slot][0] = gt;
    s_grab[slot][1] = gb;
  };
  int gs = 0;  // slot of the current grab
  if (tid == 0) grab(int(blockIdx.x % T), 0);
  __syncthreads();
  int t = s_grab[0][0];
  int b_next = s_grab[0][1];
  int b_end = b_next + CH < int(B) ? b_next + CH : int(B);
  if (b_next >= 0) build_masks(b_next, 0);
  __syncthreads();
  int mb = 0;
  uint32_t kq = 0;      // quarters stored so far (staging ring position)
  uint32_t wmask = 0u;  // this warp's rows that carry a power-of-two scale
  int64_t cur_tile = -1;
  while (b_next >= 0) {
    const int b = b_next++;
    const bool last = b_next >= b_end;  // last item of this grab
    if (last && tid == 0) grab(t, gs ^ 1);
    const int64_t i0 = int64_t(t) * TI;
    const bool ident = b == D / 2;

    if (t != cur_tile) {  // this warp's 8 rows into tensor memory, scaled, as B fragments
      wmask = 0u;
      uint32_t* scr = reinterpret_cast<uint32_t*>(smem + OFF_SCR) + warp * 512;
#pragma unroll 1
      for (int r = 0; r < RPW; ++r) {
        const int64_t row = i0 + warp * RPW + r;
        const bool rv = row < a.m;
        const float* arow = a.A + (rv ? row : 0) * a.lda;
        // lane holds p = 4 (lane + 32 c) + e, c < 8, e < 4: coalesced loads, all
        // in flight together; 16-byte loads when the row is a whole aligned d
        float x[32];
        const bool vec = rv && a.n == D && (reinterpret_cast<uintptr_t>(arow) & 15u) == 0;
        if (vec) {
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const float4 f = __ldg(reinterpret_cast<const float4*>(arow) + lane + 32 * c);
            x[4 * c] = f.x;
            x[4 * c + 1] = f.y;
            x[4 * c + 2] = f.z;
            x[4 * c + 3] = f.w;
          }
        } else {
#pragma unroll
          for (int c = 0; c < 8; ++c)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int p = 4 * (lane + 32 * c) + e;
              x[4 * c + e] = (rv && p < a.n) ? arow[p] : 0.f;
            }
        }
        float mx = 0.f;
#pragma unroll
        for (int k = 0; k < 32; ++k) mx = fmaxf(mx, fabsf(x[k]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        // rows whose largest entry lies in [2^-8, 2^6) are used as they are
        // (stage values below 2^14, 11 significant bits relative to ||a_i||);
        // others are scaled by 2^e (largest entry into [1/2, 1))
        int ex = 0;
        if (mx > 0.f) frexpf(mx, &ex);  // mx = f 2^ex, f in [1/2, 1)
        const int e = (mx > 0.f && (ex < -7 || ex > 6)) ? -ex : 0;
        const float sc = ldexpf(1.f, e);
        if (e != 0) wmask |= 1u << r;
        // the row as float16 pairs in p order, then each lane's fragment words
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          scr[2 * (lane + 32 * c)] = pack_h2(x[4 * c] * sc, x[4 * c + 1] * sc);
          scr[2 * (lane + 32 * c) + 1] = pack_h2(x[4 * c + 2] * sc, x[4 * c + 3] * sc);
        }
        __syncwarp();
        uint32_t v[16];
#pragma unroll
        for (int idx = 0; idx < 16; ++idx)  // p = 256 p2 + 16 (g + 8 nt) + 2 q + 8 j
          v[idx] = scr[128 * (idx >> 2) + 8 * (g + 8 * ((idx >> 1) & 1)) + q + 4 * (idx & 1)];
        __syncwarp();  // the next row reuses the scratch
        k10::tmem_st16(tx + uint32_t(16 * r), v);
        // second-stage A operand: W_16 times 2^-e, exact in float16 for e in
        // [-15, 24]; any remainder is undone in float32 on the outputs
        const int ef = e < -15 ? -15 : (e > 24 ? 24 : e);
        const uint32_t mag = ef <= 14 ? uint32_t(15 - ef) << 10 : 1u << (24 - ef);
        frag[(warp * RPW + r) * 32 + lane] =
            make_uint4((w16[0] & 0x80008000u) | mag | (mag << 16),
                       (w16[1] & 0x80008000u) | mag | (mag << 16),
                       (w16[2] & 0x80008000u) | mag | (mag << 16),
                       (w16[3] & 0x80008000u) | mag | (mag << 16));
        if (lane == 0) erem[warp * RPW + r] = e - ef;
      }
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      __syncwarp();
      cur_tile = t;
    }

    if (!ident) {
      // sign flip and the 4-point stage over p2, row by row, back to tensor memory
      uint32_t mk[16];
      {
        const uint4* m4 = reinterpret_cast<const uint4*>(masks + mb * MASKW);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const uint4 u = m4[c * 32 + lane];
          mk[4 * c] = u.x;
          mk[4 * c + 1] = u.y;
          mk[4 * c + 2] = u.z;
          mk[4 * c + 3] = u.w;
        }
      }
      // four rows per tensor-memory round trip: their loads are in flight together
#pragma unroll 1
      for (int r0 = 0; r0 < RPW; r0 += 4) {
        uint32_t v[4][16];
#pragma unroll
        for (int rr = 0; rr < 4; ++rr) k10::tmem_ld16(tx + uint32_t(16 * (r0 + rr)), v[rr]);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int rr = 0; rr < 4; ++rr)
          asm volatile(""
                       : "+r"(v[rr][0]), "+r"(v[rr][1]), "+r"(v[rr][2]), "+r"(v[rr][3]),
                         "+r"(v[rr][4]), "+r"(v[rr][5]), "+r"(v[rr][6]), "+r"(v[rr][7]),
                         "+r"(v[rr][8]), "+r"(v[rr][9]), "+r"(v[rr][10]), "+r"(v[rr][11]),
                         "+r"(v[rr][12]), "+r"(v[rr][13]), "+r"(v[rr][14]), "+r"(v[rr][15]));
#pragma unroll
        for (int rr = 0; rr < 4; ++rr) {
          uint32_t y[16];
#pragma unroll
          for (int c = 0; c < 4; ++c) {  // register c of each p2 unit: (nt, j)
            const uint32_t a0 = v[rr][c] ^ mk[c], a1 = v[rr][4 + c] ^ mk[4 + c];
            const uint32_t a2 = v[rr][8 + c] ^ mk[8 + c], a3 = v[rr][12 + c] ^ mk[12 + c];
            const uint32_t s01 = hadd2(a0, a1), d01 = hsub2(a0, a1);
            const uint32_t s23 = hadd2(a2, a3), d23 = hsub2(a2, a3);
            y[c] = hadd2(s01, s23);       // w2 = 0
            y[4 + c] = hadd2(d01, d23);   // w2 = 1
            y[8 + c] = hsub2(s01, s23);   // w2 = 2
            y[12 + c] = hsub2(d01, d23);  // w2 = 3
          }
          k10::tmem_st16(ty + uint32_t(16 * (r0 + rr)), y);
        }
      }
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }

    // each quarter's tensor-memory loads are issued during the previous
    // quarter (ping-pong registers), so their latency hides behind its stores
    uint32_t yq[2][RPW][4];
    if (!ident) {
#pragma unroll
      for (int r = 0; r < RPW; ++r) tmem_ld4(ty + uint32_t(16 * r), yq[0][r]);
    }
    // Quarters are staged in rounds of two (64 KiB): one proxy fence and one
    // barrier per round; the round's buffer was stored two rounds ago.
#pragma unroll
    for (int q2 = 0; q2 < 4; ++q2) {
      unsigned char* Fb = smem + size_t((kq & 1) * 2 + (q2 & 1)) * FBUF;
      if (!ident) {
        uint32_t (&yv)[RPW][4] = yq[q2 & 1];
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int r = 0; r < RPW; ++r)
          asm volatile("" : "+r"(yv[r][0]), "+r"(yv[r][1]), "+r"(yv[r][2]), "+r"(yv[r][3]));
        uint32_t out[8][4];
        float lo[8];
        // the warp's rows carry no scale in the usual case: plain W_16 then
        auto rows = [&](auto scaled_tag) {
          constexpr bool SC = decltype(scaled_tag)::value;
#pragma unroll
          for (int r = 0; r < RPW; ++r) {
            float d1[2][4];
            mma_f16(d1[0], w16, yv[r][0], yv[r][1]);  // [w0][p1 0..7]
            mma_f16(d1[1], w16, yv[r][2], yv[r][3]);  // [w0][p1 8..15]
            uint32_t fr[4] = {w16[0], w16[1], w16[2], w16[3]};
            if constexpr (SC) {
              if ((wmask >> r) & 1u) {  // this row's W_16 2^-e
                const uint4 f4 = frag[(warp * RPW + r) * 32 + lane];
                fr[0] = f4.x;
                fr[1] = f4.y;
                fr[2] = f4.z;
                fr[3] = f4.w;
              }
            }
            float d2[2][4];
            mma_f16(d2[0], fr, pack_h2(d1[0][0], d1[0][1]), pack_h2(d1[1][0], d1[1][1]));
            mma_f16(d2[1], fr, pack_h2(d1[0][2], d1[0][3]), pack_h2(d1[1][2], d1[1][3]));
            if constexpr (SC) {
              const int er = ((wmask >> r) & 1u) ? erem[warp * RPW + r] : 0;
              if (er != 0) {
                const float s2 = ldexpf(1.f, -er);
#pragma unroll
                for (int m = 0; m < 2; ++m)
#pragma unroll
                  for (int e = 0; e < 4; ++e) d2[m][e] *= s2;
              }
            }
#pragma unroll
            for (int pos = 0; pos < 8; ++pos) {
              const float val = d2[pos >> 2][pos & 3];
              if (r & 1)
                out[pos][r >> 1] = pack_b2(lo[pos], val);
              else
                lo[pos] = val;
            }
          }
        };
        if (wmask == 0u)
          rows(std::integral_constant<bool, false>{});
        else
          rows(std::integral_constant<bool, true>{});
        if (q2 < 3) {
#pragma unroll
          for (int r = 0; r < RPW; ++r)
            tmem_ld4(ty + uint32_t(16 * r + 4 * (q2 + 1)), yq[(q2 + 1) & 1][r]);
        }
        // position pos: w1 = g + 8 ((pos & 3) >> 1), w0 = 2q + 8 (pos >> 2) + (pos & 1);
        // the warp's 8 rows are 16-byte chunk `warp` ^ (w & 7) of the 128-byte
        // row w.  Lanes with odd g store their positions in pairwise swapped
        // order, so that in each quarter-warp the lanes g = 2k and 2k + 1 hit
        // different 16-byte chunks (their w differ by 16, not in w & 7).
        const bool oddg = g & 1;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int pos = i ^ int(oddg);
          const int w = 16 * (g + 8 * ((pos & 3) >> 1)) + 2 * q + 8 * (pos >> 2) + (pos & 1);
          const uint32_t addr = smem_addr(Fb + w * (TI * 2) + ((warp ^ (w & 7)) << 4));
          asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr),
                       "r"(oddg ? out[i ^ 1][0] : out[i][0]), "r"(oddg ? out[i ^ 1][1] : out[i][1]),
                       "r"(oddg ? out[i ^ 1][2] : out[i][2]), "r"(oddg ? out[i ^ 1][3] : out[i][3])
                       : "memory");
        }
      } else {
        // identity basis: R[d/2][w][i] = sqrt(d) A[i][w] straight from A; thread
        // w of the quarter reads column w of the tile's rows (a warp reads 128
        // contiguous bytes of a row per load) and packs 8 rows per store
        const int w = tid;  // THREADS == QW
        const int64_t col = int64_t(QW) * q2 + w;
#pragma unroll 1
        for (int half = 0; half < 2; ++half) {  // 32 loads in flight before the stores
          float v[TI / 2];
#pragma unroll
          for (int k = 0; k < TI / 2; ++k) {
            const int64_t row = i0 + (TI / 2) * half + k;
            v[k] = (row < a.m && col < a.n) ? 32.f * a.A[row * a.lda + col] : 0.f;
          }
#pragma unroll
          for (int c4 = 0; c4 < TI / 16; ++c4) {
            const int ch = (TI / 16) * half + c4;
            const uint32_t addr = smem_addr(Fb + w * (TI * 2) + ((ch ^ (w & 7)) << 4));
            asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr),
                         "r"(pack_b2(v[8 * c4], v[8 * c4 + 1])),
                         "r"(pack_b2(v[8 * c4 + 2], v[8 * c4 + 3])),
                         "r"(pack_b2(v[8 * c4 + 4], v[8 * c4 + 5])),
                         "r"(pack_b2(v[8 * c4 + 6], v[8 * c4 + 7]))
                         : "memory");
          }
        }
      }
      // the next basis (of this grab, or the first of the next one, which
      // thread 0 took at the start of this item and is visible after round
      // 0's barrier): its sign words are requested at quarter 2 and become
      // masks, in the other buffer, at quarter 3
      if (q2 >= 2) {
        const int nb = last ? s_grab[gs ^ 1][1] : b_next;
        if (nb >= 0) {
          if (q2 == 2)
            sign_words(nb, wd_next);
          else
            put_masks(wd_next, mb ^ 1);
        }
      }
      if ((q2 & 1) == 0) continue;  // the round's second quarter ends it
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      // the next round's buffers were stored by the previous round, whose
      // stores must be done reading them
      if (tid == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        tma_store_2d(&tmap, smem_addr(Fb - FBUF), int(i0), b * D + QW * (q2 - 1));
        tma_store_2d(&tmap, smem_addr(Fb), int(i0), b * D + QW * q2);
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      }
      ++kq;
    }
    mb ^= 1;
    if (last) {  // move to the grab taken during this item (-1: all tiles are done)
      gs ^= 1;
      t = s_grab[gs][0];
      b_next = s_grab[gs][1];
      b_end = b_next + CH < int(B) ? b_next + CH : int(B);
    }
  }
  if (tid == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
}

}  // namespace k10tc

int launch_d1024_tc(const Plan& p) {
  tc::EncodeTiledFn enc = tc::encoder();
  if (enc == nullptr) return KERDOCK_ERR_UNSUPPORTED;
  // R[b][w][i] (bfloat16) as rows (b, w) of ldr elements: box 64 rows x 256 w
  CUtensorMap map;
  const cuuint64_t dims[2] = {cuuint64_t(p.ldr), cuuint64_t(p.B) * cuuint64_t(p.d)};
  const cuuint64_t strides[1] = {cuuint64_t(p.ldr) * 2};
  const cuuint32_t box[2] = {k10tc::TI, k10tc::QW};
  const cuuint32_t es[2] = {1, 1};
  if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, p.repr, dims, strides, box, es,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
          CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return KERDOCK_ERR_UNSUPPORTED;
  auto kern = k10tc::preprocess_d1024_tc_kernel;
  KD_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   int(k10tc::SMEM)));
  PreArgs a;
  a.A = p.A;
  a.lda = p.lda;
  a.m = p.m;
  a.n = p.n;
  a.signs = p.signs();
  a.sign_words = p.sign_words;
  a.R = p.repr;
  a.ldr = p.ldr;
  a.status = p.status();
  a.num_tiles = (p.ldr + k10tc::TI - 1) / k10tc::TI;
  a.group = 1;
  if (a.num_tiles > int64_t(kWorkCounters)) return KERDOCK_ERR_UNSUPPORTED;
  a.work = p.work_counters();
  KD_CUDA_TRY(cudaMemsetAsync(a.work, 0, size_t(a.num_tiles) * sizeof(int), p.stream));
  // one CTA per SM (its shared memory and all 512 tensor-memory columns)
  int64_t grid = p.num_sms;
  const int64_t grabs = a.num_tiles * ((p.B + 7) / 8);
  if (grid > grabs) grid = grabs;
  kern<<<unsigned(grid), k10tc::THREADS, k10tc::SMEM, p.stream>>>(a, map);
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
    case 10:
      if (sizeof(OutT) == 2) return launch_d1024_tc(p);
      return launch_d1024<OutT>(p);
    case 12:
      if (sizeof(OutT) == 2) return launch_d4096_tc(p);
      return launch_d4096_tc32(p);
    default: return KERDOCK_ERR_UNSUPPORTED;
  }
}

}  // namespace

int launch_preprocess(const Plan& p) {
  return p.dtype == KERDOCK_BF16 ? launch_typed<__nv_bfloat16>(p) : launch_typed<float>(p);
}

}  // namespace kd
