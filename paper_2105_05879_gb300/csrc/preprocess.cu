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
#include <cooperative_groups.h>

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

// ---------------------------------------------------------------------------
// d = 4096: a cluster of four CTAs shares one tile of TI rows (TI = 32: the
// representation's rows then get 64-byte (bfloat16) or 128-byte (float32)
// runs per output row).  Write p = 1024 q + 64 s + j: CTA q keeps the quarter
// p in [1024 q, 1024 (q+1)) of the tile in shared memory; its thread (r, s)
// holds row r's 64 values of source s in registers and runs the six butterfly
// stages over j there (phase 1).  Output w = 64 w_hi + w_lo: the w_lo of the
// phase-1 results are spread over the cluster, CTA c taking w_lo in
// [16 c, 16 c + 16), and each CTA's thread (r, w_lo) combines the 64 sources
// (q, s) of its column in two rounds of 32 (s < 8, s >= 8), five stages per
// round plus one combining stage (phase 2).  Each round, every thread of the
// sending half writes its values straight into the owners' exchange buffers
// over distributed shared memory; split cluster barriers separate writing from
// reading, and the "buffer free" half of each barrier pair overlaps with the
// next round's arithmetic.
// ---------------------------------------------------------------------------
namespace cg = cooperative_groups;

template <int TI>
struct Big {
  static constexpr int D = 4096, Q = 1024, CL = 4;  // CTAs per cluster, p per CTA
  static constexpr int NS = 16, RG = 64;             // sources per CTA, values per source
  static constexpr int THREADS = TI * NS;            // thread (r, s) = (tid % TI, tid / TI)
  static constexpr int WLC = RG / CL;                // w_lo per CTA: 16
  static constexpr int HS = NS / 2;                  // sources per CTA per round: 8
  static constexpr int RSRC = HS * CL;               // sources per round: 32
  static constexpr int AST = Q + 4;                  // A-tile row stride (floats)
  static constexpr int XSRC = WLC * TI + (TI == 32 ? 0 : 16);  // floats per source: [w_lo][row]
  static constexpr size_t SMEM = size_t(TI) * AST * 4 + size_t(RSRC) * XSRC * 4;
  static constexpr int MINB = THREADS >= 512 ? 1 : 2;
  static_assert(THREADS <= 1024 && TI % 8 == 0, "tile");
};

__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

template <typename T>
__device__ __forceinline__ void store_one(T* dst, float v);
template <>
__device__ __forceinline__ void store_one<float>(float* dst, float v) {
  asm volatile("st.global.cs.f32 [%0], %1;" ::"l"(dst), "f"(v) : "memory");
}
template <>
__device__ __forceinline__ void store_one<__nv_bfloat16>(__nv_bfloat16* dst, float v) {
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  asm volatile("st.global.cs.b16 [%0], %1;" ::"l"(dst),
               "h"(*reinterpret_cast<const unsigned short*>(&h))
               : "memory");
}

template <typename OutT, int TI>
__global__ void __launch_bounds__(Big<TI>::THREADS, Big<TI>::MINB)
    preprocess_d4096_kernel(const PreArgs a) {
  using C = Big<TI>;
  constexpr int64_t B = C::D / 2 + 1;
  cg::cluster_group cluster = cg::this_cluster();
  const int q = int(cluster.block_rank());
  extern __shared__ __align__(16) float smem[];
  float* At = smem;                            // [TI][AST]: this CTA's quarter of the tile
  float* X = smem + size_t(TI) * C::AST;       // [32 sources][16 w_lo][TI rows]
  float* Xc[C::CL];
#pragma unroll
  for (int c = 0; c < C::CL; ++c) Xc[c] = cluster.map_shared_rank(X, c);
  OutT* R = static_cast<OutT*>(a.R);
  const int tid = threadIdx.x;
  const int r = tid % TI, s = tid / TI;  // phase 1: (row, source); phase 2: (row, w_lo in CTA)
  const float sqrt_d = 64.f;

  const ItemRange ir =
      item_range(blockIdx.x / C::CL, gridDim.x / C::CL, a.group, a.num_tiles, B);
  int64_t cur_tile = -1;
  cluster_arrive();  // pairs with the first "exchange buffers free" wait

  for (int64_t item = ir.beg; item < ir.end; ++item) {
    const int64_t tg = item / B;
    const int b = int(item - tg * B);
    const int64_t t = tg * a.group + ir.slot;
    const int64_t i0 = t * TI;
    const bool ident = b == C::D / 2;
    if (t != cur_tile) {
      __syncthreads();  // the previous tile's phase 1 is done everywhere in this CTA
      for (int idx = tid; idx < TI * C::Q; idx += C::THREADS) {
        const int i = idx / C::Q, pq = idx % C::Q;
        const int64_t gp = int64_t(q) * C::Q + pq;
        float v = 0.f;
        if (i0 + i < a.m && gp < a.n) v = a.A[(i0 + i) * a.lda + gp];
        At[i * C::AST + pq] = v;
      }
      cur_tile = t;
      __syncthreads();
    }

    // Phase 1: step (i) of Lemma 6 from the source's two sign words, then the
    // six stages over j in registers.
    uint32_t wd[2] = {0u, 0u};
    if (!ident) {
      const uint32_t* srow = a.signs + int64_t(b) * a.sign_words + q * (C::Q / 32) + s * 2;
      wd[0] = __ldg(srow);
      wd[1] = __ldg(srow + 1);
    }
    float2 v[C::RG / 2];
#pragma unroll
    for (int j = 0; j < C::RG; j += 4) {
      float4 x4 = *reinterpret_cast<const float4*>(&At[r * C::AST + s * C::RG + j]);
      if (!ident) {
        uint32_t f[4];
#pragma unroll
        for (int e = 0; e < 4; ++e)
          f[e] = (wd[(j + e) >> 5] << (31 - ((j + e) & 31))) & 0x80000000u;
        x4.x = __uint_as_float(__float_as_uint(x4.x) ^ f[0]);
        x4.y = __uint_as_float(__float_as_uint(x4.y) ^ f[1]);
        x4.z = __uint_as_float(__float_as_uint(x4.z) ^ f[2]);
        x4.w = __uint_as_float(__float_as_uint(x4.w) ^ f[3]);
      }
      v[j / 2] = make_float2(x4.x, x4.y);
      v[j / 2 + 1] = make_float2(x4.z, x4.w);
    }
    if (!ident) fwht_pairs<C::RG / 2>(v);

    // Phase 2 in two rounds of 32 sources (q', s') with s' / 8 == round.
    float2 z[2][C::RSRC / 2];  // per round: pairs (source k, source k + 16)
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      cluster_wait();  // every CTA is done reading the exchange buffers
      if ((s >> 3) == e) {
        const int src = q * C::HS + (s & 7);
#pragma unroll
        for (int j = 0; j < C::RG; ++j) {
          const float val = (j & 1) ? v[j / 2].y : v[j / 2].x;
          Xc[j / C::WLC][src * C::XSRC + (j % C::WLC) * TI + r] = val;
        }
      }
      cluster_arrive();  // this round's values are written
      cluster_wait();    // ... by every CTA of the cluster
#pragma unroll
      for (int k = 0; k < C::RSRC / 2; ++k)
        z[e][k] = make_float2(X[k * C::XSRC + s * TI + r],
                              X[(k + C::RSRC / 2) * C::XSRC + s * TI + r]);
      cluster_arrive();  // done reading; the buffers may be refilled
      if (!ident) {
#pragma unroll
        for (int k = 0; k < C::RSRC / 2; ++k)
          z[e][k] = make_float2(z[e][k].x + z[e][k].y, z[e][k].x - z[e][k].y);
        fwht_across<C::RSRC / 2>(z[e]);
      }
    }

    // Combine the rounds (source bit s / 8) and store.  Round-local source
    // k = 8 q' + (s' mod 8) and the round e give w_hi = 16 q' + 8 e + (s' mod 8).
    const int64_t row = i0 + r;
    if (row < a.ldr) {
      OutT* rb = R + (int64_t(b) * C::D + q * C::WLC + s) * a.ldr + row;
      const int64_t wstride = int64_t(C::RG) * a.ldr;  // one step of w_hi
#pragma unroll
      for (int k = 0; k < C::RSRC; ++k) {
        const float z0 = (k < C::RSRC / 2) ? z[0][k].x : z[0][k - C::RSRC / 2].y;
        const float z1 = (k < C::RSRC / 2) ? z[1][k].x : z[1][k - C::RSRC / 2].y;
        float y0, y1;
        if (ident) {
          y0 = z0 * sqrt_d;
          y1 = z1 * sqrt_d;
        } else {
          y0 = z0 + z1;
          y1 = z0 - z1;
        }
        const int whi = (k >> 3) * 16 + (k & 7);
        store_one<OutT>(rb + int64_t(whi) * wstride, y0);
        store_one<OutT>(rb + int64_t(whi + 8) * wstride, y1);
      }
    }
  }
  cluster_wait();  // pairs with the last arrive: no CTA leaves while others read its buffers
}

// Largest power of two <= limit and <= num_tiles (the tile group size G).
int64_t pick_group(int64_t num_tiles, int64_t limit) {
  int64_t g = 1;
  while (g * 2 <= limit && g * 2 <= num_tiles) g *= 2;
  return g;
}

template <typename OutT>
int launch_d4096(const Plan& p) {
  constexpr int TI = 32;
  using C = Big<TI>;
  auto kern = preprocess_d4096_kernel<OutT, TI>;
  KD_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   int(C::SMEM)));
  PreArgs a;
  a.A = p.A;
  a.lda = p.lda;
  a.m = p.m;
  a.n = p.n;
  a.signs = p.signs();
  a.sign_words = p.sign_words;
  a.R = p.repr;
  a.ldr = p.ldr;
  a.num_tiles = (p.ldr + TI - 1) / TI;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C::CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(C::THREADS);
  cfg.dynamicSmemBytes = C::SMEM;
  cfg.stream = p.stream;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3(C::CL);
  int clusters = 0;
  KD_CUDA_TRY(cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg));
  if (clusters < 1) return KERDOCK_ERR_UNSUPPORTED;
  // groups of up to 4 clusters on adjacent 32-row tiles: 4 x 64 B = two whole
  // 128-byte lines per output row for bfloat16
  a.group = pick_group(a.num_tiles, clusters < 4 ? clusters : 4);
  int64_t ngrp = clusters / a.group;
  const int64_t items = ((a.num_tiles + a.group - 1) / a.group) * p.B;
  if (ngrp > items) ngrp = items;
  cfg.gridDim = dim3(unsigned(ngrp * a.group * C::CL));
  KD_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, a));
  return KERDOCK_OK;
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

template <typename OutT>
int launch_typed(const Plan& p) {
  switch (p.k) {
    case 2: return launch_small<2, OutT>(p);
    case 4: return launch_small<4, OutT>(p);
    case 6: return launch_small<6, OutT>(p);
    case 8: return launch_small<8, OutT>(p);
    case 10: return launch_small<10, OutT>(p);
    case 12: return launch_d4096<OutT>(p);
    default: return KERDOCK_ERR_UNSUPPORTED;
  }
}

}  // namespace

int launch_preprocess(const Plan& p) {
  return p.dtype == KERDOCK_BF16 ? launch_typed<__nv_bfloat16>(p) : launch_typed<float>(p);
}

}  // namespace kd
