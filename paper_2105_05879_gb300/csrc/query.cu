// query.cu -- the streaming step of Algorithm 1 for a batch of queries.
//
// One CTA owns one query at a time (persistent grid, static round robin):
//   a3  draw l_j = floor(SplitMix64(seed + G(qN + j + 1)) * L / 2^64)
//   a4  c_j = s_{l_j}^T x: for a Kerdock basis b, sum_p (-1)^{Q_b(p)+w.p} x_p
//       (one warp per sample, lane = p mod 32, sign bits from the device
//       table); for the identity basis sqrt(d) x_w (0 when w >= n)
//   a5  ybar_k = (1/J) sum_{j in batch k} c_j R[l_j][.]: rows of the
//       representation stream through a shared-memory ring filled by the TMA
//       engine (cp.async.bulk, one whole row per copy, mbarrier completion);
//       each thread owns fixed 16-byte column granules, so the sum order is
//       fixed and the result deterministic
//   a6  mu_i = median_k ybar_{k,i} (mean of the two middle values for even K)
//   a7  the S indices of largest |mu_i| (radix select on the float bits,
//       ties to the smaller index), in ascending order
//   a8  v_i = a_i^T x for the selected rows, keep |v_i| >= eps, compact.
// Theorem 3 gives the estimator, Algorithm 1 the steps, Sec. 4 the top-10s
// refinement.
#include "kerdock_internal.cuh"

namespace kd {
namespace {

constexpr int kQThreads = 256;
constexpr int kQWarps = kQThreads / 32;
constexpr int kMaxSlots = 32;
constexpr int kChunk = 1024;           // samples drawn and weighted per round
constexpr size_t kRingTarget = 64 << 10;  // bytes of representation rows in flight per CTA
constexpr size_t kMeansSmemMax = 32 << 10;
constexpr int kMaxCtasPerSm = 2;

struct QueryArgs {
  const void* R;
  const uint32_t* signs;
  int64_t sign_words;
  const float* A;
  int64_t lda;
  const float* X;
  int64_t ldx;
  int64_t Q, m, n, d, L, ldr, N;
  int k, J, K, S;
  float eps, inv_J, sqrt_d;
  uint64_t seed;
  int flags;
  int a_vec4;  // rows of A are 16-byte aligned and n % 4 == 0
  int nslot;
  uint32_t row_bytes;
  // dynamic shared-memory layout (byte offsets)
  uint32_t off_xs, off_ells, off_coefs, off_means;
  float* means_gmem;  // non-null when the batch means live in the workspace
  int32_t* out_idx;
  float* out_val;
  int32_t* out_count;
  float* mu_out;
  int64_t* ells_out;
  float* coef_out;
  uint32_t* status;
};

template <typename RT>
struct Granule;
template <>
struct Granule<float> {
  static constexpr int kElems = 4;
  __device__ static void load(const unsigned char* p, float (&o)[4]) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x;
    o[1] = v.y;
    o[2] = v.z;
    o[3] = v.w;
  }
};
template <>
struct Granule<__nv_bfloat16> {
  static constexpr int kElems = 8;
  __device__ static void load(const unsigned char* p, float (&o)[8]) {
    const uint4 v = *reinterpret_cast<const uint4*>(p);
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[e]));
      o[2 * e] = f.x;
      o[2 * e + 1] = f.y;
    }
  }
};

// Exclusive prefix sum over the CTA; *total receives the sum of all v.
__device__ __forceinline__ int block_exclusive_scan(int v, int* scratch, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) scratch[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int s = lane < kQWarps ? scratch[lane] : 0;
#pragma unroll
    for (int o = 1; o < kQWarps; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < kQWarps) scratch[lane] = s;
  }
  __syncthreads();
  const int before = warp > 0 ? scratch[warp - 1] : 0;
  *total = scratch[kQWarps - 1];
  __syncthreads();
  return before + x - v;
}

// 32x32 bit-matrix transpose across a warp: on entry lane L holds row L
// (bit t = entry (L, t)); on exit lane L holds column L (bit t = entry (t, L)).
// Recursive exchange of off-diagonal blocks of size 16, 8, 4, 2, 1.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t v, int lane) {
  const uint32_t lo_masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const int j = 16 >> i;
    const uint32_t m = lo_masks[i];
    const uint32_t t = __shfl_xor_sync(0xffffffffu, v, j);
    v = (lane & j) ? ((v & ~m) | ((t >> j) & m)) : ((v & m) | ((t & m) << j));
  }
  return v;
}

// c = s_l^T x for a Kerdock sample l = (b, w): sum over p < n of
// (-1)^{Q_b(p) + w.p} x_p.  Lane L owns p = 32 t + L.  The sign bits of basis b
// for 32 consecutive words are transposed so that lane L holds, in one
// register, the bits of its own p for 32 values of t; the Walsh character
// (-1)^{w.p} splits into a per-lane part (-1)^{(w mod 32).L} and a per-t part
// (-1)^{(w >> 5).t}, both folded into that register.  x comes from registers
// (XREG, n <= 1024: xr[t] = x_{32t+L}) or from shared memory.
template <bool XREG>
__device__ __forceinline__ float kerdock_coefficient(const uint32_t* __restrict__ srow,
                                                     int nwords, uint32_t w, int lane,
                                                     const float (&xr)[32],
                                                     const float* __restrict__ xs) {
  const uint32_t whi = w >> 5;
  const uint32_t pl = __popc(w & 31u & uint32_t(lane)) & 1u;
  // bit t of wmask = parity(whi & t) for t < 32
  const uint32_t wmask = __ballot_sync(0xffffffffu, __popc(whi & 31u & uint32_t(lane)) & 1u);
  float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, acc3 = 0.f;
  const int groups = (nwords + 31) >> 5;
  for (int g = 0; g < groups; ++g) {
    const int t0 = g << 5;
    const uint32_t word = t0 + lane < nwords ? __ldg(srow + t0 + lane) : 0u;
    uint32_t F = warp_transpose32(word, lane) ^ wmask;
    if ((__popc(whi & uint32_t(t0)) & 1u) ^ pl) F = ~F;
#pragma unroll
    for (int t = 0; t < 32; t += 4) {
      const float x0 = XREG ? xr[t] : xs[(t0 + t) * 32 + lane];
      const float x1 = XREG ? xr[t + 1] : xs[(t0 + t + 1) * 32 + lane];
      const float x2 = XREG ? xr[t + 2] : xs[(t0 + t + 2) * 32 + lane];
      const float x3 = XREG ? xr[t + 3] : xs[(t0 + t + 3) * 32 + lane];
      acc0 += __uint_as_float(__float_as_uint(x0) ^ ((F << (31 - t)) & 0x80000000u));
      acc1 += __uint_as_float(__float_as_uint(x1) ^ ((F << (30 - t)) & 0x80000000u));
      acc2 += __uint_as_float(__float_as_uint(x2) ^ ((F << (29 - t)) & 0x80000000u));
      acc3 += __uint_as_float(__float_as_uint(x3) ^ ((F << (28 - t)) & 0x80000000u));
    }
  }
  return warp_sum((acc0 + acc1) + (acc2 + acc3));
}

__device__ __forceinline__ uint32_t abs_key(float v) { return __float_as_uint(v) & 0x7fffffffu; }

template <typename RT, int GPT, bool XREG>
__global__ void __launch_bounds__(kQThreads, 2) query_kernel(const QueryArgs a) {
  using G = Granule<RT>;
  constexpr int GR = G::kElems;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t full_bar[kMaxSlots];
  __shared__ __align__(8) uint64_t empty_bar[kMaxSlots];
  __shared__ int s_scan[kQWarps];
  __shared__ uint32_t s_hist[256];
  __shared__ uint32_t s_digit, s_remaining;
  __shared__ int s_abort;

  unsigned char* ring = smem;
  float* xs = reinterpret_cast<float*>(smem + a.off_xs);
  int32_t* ells = reinterpret_cast<int32_t*>(smem + a.off_ells);
  float* coefs = reinterpret_cast<float*>(smem + a.off_coefs);
  float* means = a.means_gmem != nullptr
                     ? a.means_gmem + int64_t(blockIdx.x) * a.K * a.ldr
                     : reinterpret_cast<float*>(smem + a.off_means);
  // After the gather the ring is reused for mu, the selection and its values.
  float* mus = reinterpret_cast<float*>(smem);
  int32_t* sel = reinterpret_cast<int32_t*>(smem + a.ldr * 4);
  float* vals = reinterpret_cast<float*>(smem + a.ldr * 4 + ((a.S + 3) / 4 * 4) * 4);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const RT* R = static_cast<const RT*>(a.R);
  const int64_t xpad = a.d > 32 ? a.d : 32;
  const int nwords = int((a.n + 31) / 32);
  const int64_t half = a.d / 2;

  if (tid == 0) {
    for (int s = 0; s < a.nslot; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], kQWarps);
    }
    s_abort = 0;
    fence_mbar_init();
  }
  __syncthreads();

  // Ring bookkeeping: slot index and phase parity of the next row to issue
  // (thread 0 only) and of the next row to consume (every thread).
  uint32_t is_slot = 0, is_phase = 0, is_uses = 0;
  uint32_t cs_slot = 0, cs_phase = 0;

  // Thread 0 only: put the row of sample jj of the current chunk in flight.
  auto issue = [&](int jj) {
    if (is_uses >= uint32_t(a.nslot) &&
        !mbar_wait_bounded(&empty_bar[is_slot], is_phase ^ 1u)) {
      set_status(a.status, kStatusTimeout);
      s_abort = 1;
    }
    mbar_arrive_expect_tx(&full_bar[is_slot], a.row_bytes);
    const int64_t ell = ells[jj];
    bulk_g2s(ring + size_t(is_slot) * a.row_bytes, R + ell * a.ldr, a.row_bytes,
             &full_bar[is_slot]);
    ++is_uses;
    if (++is_slot == uint32_t(a.nslot)) {
      is_slot = 0;
      is_phase ^= 1u;
    }
  };

  for (int64_t q = blockIdx.x; q < a.Q; q += gridDim.x) {
    // x into shared memory, zero-padded.
    for (int64_t p = tid; p < xpad; p += kQThreads) xs[p] = p < a.n ? a.X[q * a.ldx + p] : 0.f;
    __syncthreads();
    float xr[32];
#pragma unroll
    for (int t = 0; t < 32; ++t) xr[t] = (XREG && t * 32 < xpad) ? xs[t * 32 + lane] : 0.f;
    int batch_left = a.J;  // samples left in the current batch
    int batch_idx = 0;

    float acc[GPT][GR];
#pragma unroll
    for (int u = 0; u < GPT; ++u)
#pragma unroll
      for (int e = 0; e < GR; ++e) acc[u][e] = 0.f;

    for (int64_t j0 = 0; j0 < a.N; j0 += kChunk) {
      const int cnt = int(a.N - j0 < kChunk ? a.N - j0 : kChunk);
      // a3: draw this chunk's indices.
      for (int jj = tid; jj < cnt; jj += kQThreads) {
        const uint64_t ell = sample_index(a.seed, uint64_t(q) * a.N + j0 + jj, uint64_t(a.L));
        ells[jj] = int32_t(ell);
        if (a.ells_out) a.ells_out[q * a.N + j0 + jj] = int64_t(ell);
      }
      __syncthreads();
      // Start the first rows streaming while the coefficients are computed.
      if (tid == 0) {
        const int pre = cnt < a.nslot ? cnt : a.nslot;
        for (int jj = 0; jj < pre; ++jj) issue(jj);
      }
      // a4: one warp per sample.
      for (int jj = warp; jj < cnt; jj += kQWarps) {
        const int64_t ell = ells[jj];
        const int64_t b = ell >> a.k;
        const uint32_t w = uint32_t(ell & (a.d - 1));
        float c;
        if (b == half) {
          c = w < a.n ? a.sqrt_d * xs[w] : 0.f;
        } else {
          c = kerdock_coefficient<XREG>(a.signs + b * a.sign_words, nwords, w, lane, xr, xs);
        }
        if (lane == 0) {
          coefs[jj] = c;
          if (a.coef_out) a.coef_out[q * a.N + j0 + jj] = c;
        }
      }
      __syncthreads();
      // a5: gather-accumulate.
      for (int jj = 0; jj < cnt; ++jj) {
        if (!mbar_wait_bounded(&full_bar[cs_slot], cs_phase)) {
          set_status(a.status, kStatusTimeout);
          s_abort = 1;
        }
        const float c = coefs[jj];
        const unsigned char* row = ring + size_t(cs_slot) * a.row_bytes;
#pragma unroll
        for (int u2 = 0; u2 < GPT; ++u2) {
          const int gi = tid + u2 * kQThreads;
          if (gi * GR < a.ldr) {
            float v[GR];
            G::load(row + size_t(gi) * 16, v);
#pragma unroll
            for (int e = 0; e < GR; ++e) acc[u2][e] = fmaf(c, v[e], acc[u2][e]);
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty_bar[cs_slot]);
        if (++cs_slot == uint32_t(a.nslot)) {
          cs_slot = 0;
          cs_phase ^= 1u;
        }
        if (--batch_left == 0) {  // batch batch_idx complete
          float* mrow = means + int64_t(batch_idx) * a.ldr;
#pragma unroll
          for (int u2 = 0; u2 < GPT; ++u2) {
            const int gi = tid + u2 * kQThreads;
            if (gi * GR < a.ldr) {
#pragma unroll
              for (int e = 0; e < GR; ++e) {
                mrow[gi * GR + e] = acc[u2][e] * a.inv_J;
                acc[u2][e] = 0.f;
              }
            }
          }
          batch_left = a.J;
          ++batch_idx;
        }
        if (tid == 0 && jj >= 1 && jj - 1 + a.nslot < cnt) issue(jj - 1 + a.nslot);
      }
      __syncthreads();
      if (s_abort) return;
    }

    // a6: median over the K batch means (thread-owned columns).
#pragma unroll
    for (int u2 = 0; u2 < GPT; ++u2) {
      const int gi = tid + u2 * kQThreads;
      for (int e = 0; e < GR; ++e) {
        const int64_t col = int64_t(gi) * GR + e;
        if (col >= a.ldr) break;
        float med;
        if (a.K == 1) {
          med = means[col];
        } else if (a.K == 2) {
          med = 0.5f * (means[col] + means[a.ldr + col]);
        } else {
          float v[kMaxK];
#pragma unroll
          for (int kk = 0; kk < kMaxK; ++kk) v[kk] = kk < a.K ? means[kk * a.ldr + col] : 0.f;
          const int r_lo = (a.K - 1) / 2, r_hi = a.K / 2;
          float lo = 0.f, hi = 0.f;
#pragma unroll
          for (int i = 0; i < kMaxK; ++i) {
            if (i >= a.K) break;
            int rank = 0;
#pragma unroll
            for (int j = 0; j < kMaxK; ++j)
              if (j < a.K && (v[j] < v[i] || (v[j] == v[i] && j < i))) ++rank;
            if (rank == r_lo) lo = v[i];
            if (rank == r_hi) hi = v[i];
          }
          med = (a.K & 1) ? lo : 0.5f * (lo + hi);
        }
        mus[col] = med;
        if (a.mu_out && col < a.m) a.mu_out[q * a.m + col] = med;
      }
    }
    __syncthreads();

    // a7: top-S by radix select on |mu| (4 digits of 8 bits, high first).
    const int m = int(a.m);
    uint32_t prefix = 0, mask = 0;
    uint32_t remaining = uint32_t(a.S);
    for (int pass = 0; pass < 4; ++pass) {
      const int shift = 24 - 8 * pass;
      s_hist[tid] = 0;
      __syncthreads();
      for (int i = tid; i < m; i += kQThreads) {
        const uint32_t key = abs_key(mus[i]);
        if ((key & mask) == prefix) atomicAdd(&s_hist[(key >> shift) & 255u], 1u);
      }
      __syncthreads();
      if (warp == 0) {
        const int base = (31 - lane) * 8;  // lane 0 holds the highest digits
        uint32_t sum = 0;
#pragma unroll
        for (int j2 = 0; j2 < 8; ++j2) sum += s_hist[base + j2];
        uint32_t incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += y;
        }
        const uint32_t excl = incl - sum;
        const uint32_t hit = __ballot_sync(0xffffffffu, excl < remaining && remaining <= incl);
        if (lane == __ffs(hit) - 1) {
          uint32_t cum = excl;
          for (int j2 = 7; j2 >= 0; --j2) {
            const uint32_t h = s_hist[base + j2];
            if (cum + h >= remaining) {
              s_digit = uint32_t(base + j2);
              s_remaining = remaining - cum;
              break;
            }
            cum += h;
          }
        }
      }
      __syncthreads();
      prefix |= s_digit << shift;
      mask |= 255u << shift;
      remaining = s_remaining;
      __syncthreads();
    }
    const uint32_t T = prefix;  // the S-th largest key; take `remaining` keys equal to T
    {
      const int seg = (m + kQThreads - 1) / kQThreads;
      const int lo = tid * seg, hi = lo + seg < m ? lo + seg : m;
      int eq = 0;
      for (int i = lo; i < hi; ++i) eq += abs_key(mus[i]) == T;
      int tot;
      int eq_rank = block_exclusive_scan(eq, s_scan, &tot);
      int take = 0;
      for (int i = lo; i < hi; ++i) {
        const uint32_t key = abs_key(mus[i]);
        if (key > T) {
          ++take;
        } else if (key == T) {
          take += uint32_t(eq_rank) < remaining;
          ++eq_rank;
        }
      }
      int pos = block_exclusive_scan(take, s_scan, &tot);
      eq_rank -= eq;
      for (int i = lo; i < hi; ++i) {
        const uint32_t key = abs_key(mus[i]);
        bool t2 = false;
        if (key > T) {
          t2 = true;
        } else if (key == T) {
          t2 = uint32_t(eq_rank) < remaining;
          ++eq_rank;
        }
        if (t2) sel[pos++] = i;
      }
    }
    __syncthreads();

    // a8: exact refinement v_i = a_i^T x, four rows per warp in flight.
    for (int r0 = warp * 4; r0 < a.S; r0 += kQWarps * 4) {
      float racc[4] = {0.f, 0.f, 0.f, 0.f};
      const float* arow[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) arow[u] = a.A + int64_t(sel[r0 + u < a.S ? r0 + u : r0]) * a.lda;
      if (a.a_vec4) {
        const float4* xs4 = reinterpret_cast<const float4*>(xs);
        const int n4 = int(a.n >> 2);
#pragma unroll 2
        for (int p4 = lane; p4 < n4; p4 += 32) {
          const float4 xv = xs4[p4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float4 av = __ldg(reinterpret_cast<const float4*>(arow[u]) + p4);
            racc[u] = fmaf(av.x, xv.x, racc[u]);
            racc[u] = fmaf(av.y, xv.y, racc[u]);
            racc[u] = fmaf(av.z, xv.z, racc[u]);
            racc[u] = fmaf(av.w, xv.w, racc[u]);
          }
        }
      } else {
#pragma unroll 4
        for (int64_t p = lane; p < a.n; p += 32) {
          const float xv = xs[p];
#pragma unroll
          for (int u = 0; u < 4; ++u) racc[u] = fmaf(__ldg(arow[u] + p), xv, racc[u]);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float v = warp_sum(racc[u]);
        if (lane == 0 && r0 + u < a.S) vals[r0 + u] = v;
      }
    }
    __syncthreads();
    {
      const int seg = (a.S + kQThreads - 1) / kQThreads;
      const int lo = tid * seg, hi = lo + seg < a.S ? lo + seg : a.S;
      const bool full = a.flags & KERDOCK_FLAG_FULL_OUTPUT;
      int keep = 0;
      for (int r = lo; r < hi; ++r) keep += full || fabsf(vals[r]) >= a.eps;
      int tot;
      int pos = block_exclusive_scan(keep, s_scan, &tot);
      const int64_t obase = q * a.S;
      for (int r = lo; r < hi; ++r) {
        if (full || fabsf(vals[r]) >= a.eps) {
          a.out_idx[obase + pos] = sel[r];
          a.out_val[obase + pos] = vals[r];
          ++pos;
        }
      }
      if (tid == 0) a.out_count[q] = tot;
    }
    // The ring area was written through the generic proxy (mu, selection,
    // values); order those writes before the next query's TMA writes.
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
  }
}

struct Layout {
  int nslot;
  uint32_t row_bytes;
  size_t ring, off_xs, off_ells, off_coefs, off_means, total;
  bool means_in_smem;
};

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

Layout make_layout(const Plan& p) {
  Layout L{};
  L.row_bytes = uint32_t(p.ldr * p.elem_bytes());
  int ns = int(kRingTarget / L.row_bytes);
  ns = ns < 2 ? 2 : ns > kMaxSlots ? kMaxSlots : ns;
  L.nslot = ns;
  const size_t spad = align_up(size_t(p.S), 4);
  size_t ring = size_t(ns) * L.row_bytes;
  const size_t post = size_t(p.ldr) * 4 + 2 * spad * 4;  // mu, sel, vals
  if (post > ring) ring = post;
  L.ring = align_up(ring, 128);
  L.off_xs = L.ring;
  const size_t xpad = size_t(p.d > 32 ? p.d : 32);
  L.off_ells = align_up(L.off_xs + xpad * 4, 16);
  L.off_coefs = L.off_ells + size_t(kChunk) * 4;
  L.off_means = align_up(L.off_coefs + size_t(kChunk) * 4, 16);
  const size_t means_bytes = size_t(p.K) * size_t(p.ldr) * 4;
  L.means_in_smem = means_bytes <= kMeansSmemMax;
  L.total = L.off_means + (L.means_in_smem ? means_bytes : 0);
  return L;
}

template <typename RT, int GPT, bool XREG>
int launch_typed(const Plan& p, const Layout& L, QueryArgs& a, void* ws) {
  auto kern = query_kernel<RT, GPT, XREG>;
  KD_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   int(L.total)));
  int occ = 0;
  KD_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kQThreads, L.total));
  if (occ < 1) return KERDOCK_ERR_UNSUPPORTED;
  if (occ > kMaxCtasPerSm) occ = kMaxCtasPerSm;
  int64_t grid = int64_t(p.num_sms) * occ;
  if (grid > a.Q) grid = a.Q;
  a.means_gmem = L.means_in_smem ? nullptr : static_cast<float*>(ws);
  kern<<<unsigned(grid), kQThreads, L.total, p.stream>>>(a);
  KD_CUDA_TRY(cudaGetLastError());
  return KERDOCK_OK;
}

}  // namespace

size_t apply_workspace_bytes(const Plan& p, int64_t q) {
  const Layout L = make_layout(p);
  if (L.means_in_smem || q == 0) return 0;
  return size_t(p.num_sms > 0 ? p.num_sms : 160) * kMaxCtasPerSm * size_t(p.K) * size_t(p.ldr) * 4;
}

int launch_apply(const Plan& p, const float* X, int64_t q, int64_t ldx, float eps, uint64_t seed,
                 int flags, int32_t* out_idx, float* out_val, int32_t* out_count, void* ws,
                 size_t ws_bytes, float* mu_out, int64_t* ells_out, float* coef_out) {
  (void)ws_bytes;
  const Layout L = make_layout(p);
  QueryArgs a{};
  a.R = p.repr;
  a.signs = p.signs();
  a.sign_words = p.sign_words;
  a.A = p.A;
  a.lda = p.lda;
  a.X = X;
  a.ldx = ldx;
  a.Q = q;
  a.m = p.m;
  a.n = p.n;
  a.d = p.d;
  a.L = p.L;
  a.ldr = p.ldr;
  a.N = p.N;
  a.k = p.k;
  a.J = p.J;
  a.K = p.K;
  a.S = p.S;
  a.eps = eps;
  a.inv_J = 1.0f / float(p.J);
  a.sqrt_d = float(int64_t(1) << (p.k / 2));
  a.seed = seed;
  a.flags = flags;
  a.a_vec4 = (p.n % 4 == 0 && p.lda % 4 == 0 && (reinterpret_cast<uintptr_t>(p.A) & 15) == 0) ? 1 : 0;
  a.nslot = L.nslot;
  a.row_bytes = L.row_bytes;
  a.off_xs = uint32_t(L.off_xs);
  a.off_ells = uint32_t(L.off_ells);
  a.off_coefs = uint32_t(L.off_coefs);
  a.off_means = uint32_t(L.off_means);
  a.out_idx = out_idx;
  a.out_val = out_val;
  a.out_count = out_count;
  a.mu_out = mu_out;
  a.ells_out = ells_out;
  a.coef_out = coef_out;
  a.status = p.status();
  const int64_t granule = 16 / int64_t(p.elem_bytes());
  const int64_t gpt = (p.ldr / granule + kQThreads - 1) / kQThreads;
  const bool xreg = p.n <= 1024;
  if (p.dtype == KERDOCK_BF16) {
    if (gpt <= 1) return xreg ? launch_typed<__nv_bfloat16, 1, true>(p, L, a, ws)
                              : launch_typed<__nv_bfloat16, 1, false>(p, L, a, ws);
    if (gpt <= 2) return xreg ? launch_typed<__nv_bfloat16, 2, true>(p, L, a, ws)
                              : launch_typed<__nv_bfloat16, 2, false>(p, L, a, ws);
    return launch_typed<__nv_bfloat16, 4, false>(p, L, a, ws);
  }
  if (gpt <= 1) return xreg ? launch_typed<float, 1, true>(p, L, a, ws)
                            : launch_typed<float, 1, false>(p, L, a, ws);
  if (gpt <= 2) return xreg ? launch_typed<float, 2, true>(p, L, a, ws)
                            : launch_typed<float, 2, false>(p, L, a, ws);
  return launch_typed<float, 4, false>(p, L, a, ws);
}

}  // namespace kd
