// query.cu -- the streaming step of Algorithm 1 for a batch of queries.
//
// Per query x (Algorithm 1, streaming step; Theorem 3; Sec. 4 top-10s):
//   a3  draw l_j = floor(SplitMix64(seed + G(qN + j + 1)) * L / 2^64), j < N = JK
//   a4  c_j = s_{l_j}^T x: for a Kerdock basis b, sum_p (-1)^{Q_b(p)+w.p} x_p;
//       for the identity basis sqrt(d) x_w (0 when w >= n)
//   a5  ybar_k = (1/J) sum_{j in batch k} c_j R[l_j][.]
//   a6  mu_i = median_k ybar_{k,i} (mean of the two middle values for even K)
//   a7  the S indices of largest |mu_i| (ties to the smaller index), ascending
//   a8  v_i = a_i^T x for the selected rows, keep |v_i| >= eps, compact.
//
// Kernel design: a persistent, warp-specialised CTA per SM works through its
// queries as one continuous stream of samples, so that the representation rows
// (the HBM stream that bounds the method) never stop flowing:
//   warp 0        producer: each lane draws one l_j and issues the TMA bulk
//                 copy of the row R[l_j][0..m) into its own ring slot, so one
//                 warp instruction puts up to 32 rows in flight; it also loads
//                 x of upcoming queries.
//   warps 1..3    coefficient warps: draw the same l_j themselves and compute
//                 c_j for blocks of four samples at a time from the
//                 lane-transposed sign table and x, ahead of the gather.
//   warps 4..11   gather warps: each thread owns fixed 16-byte column granules
//                 and accumulates c_j R[l_j] in registers in sample order (a
//                 fixed, deterministic summation order); batch means go to a
//                 double-buffered means area.
//   warps 12..15  finalizer warps: median, top-S radix select, exact
//                 refinement, threshold and output of the previous query while
//                 the gather warps already stream the next one.
// All hand-offs are mbarrier phases; every wait is bounded and a timeout sets
// the plan's status word and ends the CTA.
#include <mutex>

#include "kerdock_internal.cuh"

namespace kd {
namespace {

constexpr int kCoefWarps = 3;
constexpr int kGatherWarps = 8;
constexpr int kFinalWarps = 4;
constexpr int kFirstCoefWarp = 1;
constexpr int kFirstGatherWarp = kFirstCoefWarp + kCoefWarps;
constexpr int kFirstFinalWarp = kFirstGatherWarp + kGatherWarps;
constexpr int kWarps = kFirstFinalWarp + kFinalWarps;  // 16
constexpr int kThreads = kWarps * 32;                   // 512
constexpr int kGatherThreads = kGatherWarps * 32;
constexpr int kFinalThreads = kFinalWarps * 32;
constexpr int kMaxSlots = 64;  // ring rows
constexpr int kMaxChunks = 64;
constexpr int kMinChunks = 4;  // > kCoefWarps: each coefficient warp steps kCoefWarps chunks
constexpr int kXBufs = 3;
constexpr int kMBufs = 2;
constexpr int kFinalBarrier = 1;  // named barrier id of the finalizer warps
constexpr size_t kSmemBudget = 227 * 1024 - 4096;  // dynamic bytes (static ~3 KB)
constexpr size_t kRingCap = 160 * 1024;
constexpr size_t kMeansSmemMax = 64 * 1024;

struct QueryArgs {
  const void* R;
  const uint32_t* tsigns;  // lane-transposed sign table
  int64_t tsign_stride;    // words per basis in it
  const float* A;
  int64_t lda;
  const float* X;
  int64_t ldx;
  int64_t Q, m, n, d, L, ldr, N, xpad;
  int k, J, K, S;
  float eps, inv_J, sqrt_d;
  uint64_t seed;
  int flags;
  int a_vec4;  // rows of A are 16-byte aligned and n % 4 == 0
  int nchunk;   // ring chunks; each holds chunk_rows consecutive samples of one query
  int crows;    // rows per chunk (1, 2 or 4)
  int pgroup;   // chunks the producer fills per warp instruction (pgroup * crows <= 32)
  uint32_t row_bytes;
  // dynamic shared-memory layout (byte offsets)
  uint32_t off_coef, off_x, off_means, off_mu, off_sel, off_vals;
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

__device__ __forceinline__ void named_barrier_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Exclusive prefix sum over the finalizer warps; *total = sum of all v.
__device__ __forceinline__ int final_exclusive_scan(int v, int* scratch, int* total) {
  const int lane = threadIdx.x & 31;
  const int fw = (threadIdx.x >> 5) - kFirstFinalWarp;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) scratch[fw] = x;
  named_barrier_sync(kFinalBarrier, kFinalThreads);
  int before = 0, tot = 0;
#pragma unroll
  for (int w = 0; w < kFinalWarps; ++w) {
    const int s = scratch[w];
    if (w < fw) before += s;
    tot += s;
  }
  *total = tot;
  named_barrier_sync(kFinalBarrier, kFinalThreads);
  return before + x - v;
}

__device__ __forceinline__ uint32_t abs_key(float v) { return __float_as_uint(v) & 0x7fffffffu; }

// Coefficients c = s_l^T x of up to four Kerdock samples l = (b, w) at once:
// c = sum over p < n of (-1)^{Q_b(p) + w.p} x_p.  Lane L owns p = 32 t + L.
// The lane-transposed table gives lane L, in one word per 1024 values of p,
// the bits Q_b(32 t + L) for 32 values of t; the Walsh character (-1)^{w.p}
// splits into a per-lane part (-1)^{(w mod 32).L} and a per-t part
// (-1)^{(w >> 5).t}, both folded into that word.  Four samples are processed
// together so that their loads, sums and warp reductions overlap.  x comes
// from registers (XREG, n <= 1024: xr[t] = x_{32t+L}) or from shared memory.
template <bool XREG>
__device__ __forceinline__ void kerdock_coefficients4(const uint32_t* __restrict__ tsigns,
                                                      int64_t tstride, const uint32_t (&ell)[4],
                                                      int kbits, uint32_t dmask, int groups,
                                                      int lane, const float (&xr)[32],
                                                      const float* xs, float (&c)[4]) {
  float part[4] = {0.f, 0.f, 0.f, 0.f};
  uint32_t whi[4], pl[4], wmask[4];
  const uint32_t* rows[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const uint32_t w = ell[s] & dmask;
    whi[s] = w >> 5;
    pl[s] = __popc(w & 31u & uint32_t(lane)) & 1u;
    wmask[s] = __ballot_sync(0xffffffffu, __popc(whi[s] & 31u & uint32_t(lane)) & 1u);
    // identity-basis samples (b = d/2) read row d/2 - 1; their result is replaced
    const uint32_t b = ell[s] >> kbits;
    const uint32_t bmax = (dmask + 1u) / 2u - 1u;
    rows[s] = tsigns + int64_t(b < bmax ? b : bmax) * tstride;
  }
  for (int g = 0; g < groups; ++g) {
    uint32_t F[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) F[s] = __ldg(rows[s] + (g << 5) + lane);
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      F[s] ^= wmask[s];
      if ((__popc(whi[s] & uint32_t(g << 5)) & 1u) ^ pl[s]) F[s] = ~F[s];
    }
#pragma unroll
    for (int t = 0; t < 32; ++t) {
      const float xv = XREG ? xr[t] : xs[((g << 5) + t) * 32 + lane];
#pragma unroll
      for (int s = 0; s < 4; ++s)
        part[s] += __uint_as_float(__float_as_uint(xv) ^ ((F[s] << (31 - t)) & 0x80000000u));
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int s = 0; s < 4; ++s) part[s] += __shfl_xor_sync(0xffffffffu, part[s], o);
#pragma unroll
  for (int s = 0; s < 4; ++s) c[s] = part[s];
}

struct Shared {
  uint64_t row_full[kMaxChunks];
  uint64_t coef_full[kMaxChunks];
  uint64_t slot_empty[kMaxChunks];
  uint64_t x_full[kXBufs];
  uint64_t x_empty[kXBufs];
  uint64_t means_full[kMBufs];
  uint64_t means_empty[kMBufs];
  uint32_t hist[256];
  int scan[kFinalWarps];
  uint32_t digit, remaining;
  int abort_flag;
};

// Bounded wait that also gives up once another role has aborted.
__device__ __forceinline__ bool wait_phase(uint64_t* bar, uint32_t parity, Shared& sh,
                                           uint32_t* status) {
  for (uint32_t it = 0;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 255u) {
      if (*reinterpret_cast<volatile int*>(&sh.abort_flag)) return false;
      if (it > (1u << 22)) {
        set_status(status, kStatusTimeout);
        *reinterpret_cast<volatile int*>(&sh.abort_flag) = 1;
        return false;
      }
    }
  }
}

template <typename RT, int GPT, bool XREG>
__global__ void __launch_bounds__(kThreads, 1) query_kernel(const QueryArgs a) {
  using G = Granule<RT>;
  constexpr int GR = G::kElems;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ Shared sh;

  unsigned char* ring = smem;
  float* coef_s = reinterpret_cast<float*>(smem + a.off_coef);
  float* xbuf = reinterpret_cast<float*>(smem + a.off_x);
  float* means_base = a.means_gmem != nullptr
                          ? a.means_gmem + int64_t(blockIdx.x) * kMBufs * a.K * a.ldr
                          : reinterpret_cast<float*>(smem + a.off_means);
  float* mus = reinterpret_cast<float*>(smem + a.off_mu);
  int32_t* sel = reinterpret_cast<int32_t*>(smem + a.off_sel);
  float* vals = reinterpret_cast<float*>(smem + a.off_vals);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const RT* R = static_cast<const RT*>(a.R);
  const int64_t half = a.d / 2;
  const uint32_t nchunk = uint32_t(a.nchunk);
  const int CR = a.crows;
  const int64_t qchunks = (a.N + CR - 1) / CR;  // chunks per query

  if (tid == 0) {
    for (int s = 0; s < a.nchunk; ++s) {
      mbar_init(&sh.row_full[s], uint32_t(CR));
      mbar_init(&sh.coef_full[s], 1);
      mbar_init(&sh.slot_empty[s], kGatherWarps);
    }
    for (int b = 0; b < kXBufs; ++b) {
      mbar_init(&sh.x_full[b], 1);
      mbar_init(&sh.x_empty[b], kCoefWarps + 1);
    }
    for (int b = 0; b < kMBufs; ++b) {
      mbar_init(&sh.means_full[b], kGatherWarps);
      mbar_init(&sh.means_empty[b], 1);
    }
    sh.abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    uint32_t cslot = 0, cphase = 0;  // ring chunk of the next chunk to fill and its phase
    uint64_t filled = 0;             // chunks filled so far
    const int ci = lane / CR, r = lane % CR;
    int qs = 0;
    for (int64_t q = blockIdx.x; q < a.Q; q += gridDim.x, ++qs) {
      const int xb = qs % kXBufs;
      if (qs >= kXBufs &&
          !wait_phase(&sh.x_empty[xb], uint32_t(qs / kXBufs - 1) & 1u, sh, a.status))
        return;
      float* xq = xbuf + xb * a.xpad;
      for (int64_t p = lane; p < a.xpad; p += 32) xq[p] = p < a.n ? a.X[q * a.ldx + p] : 0.f;
      __syncwarp();
      if (lane == 0) mbar_arrive(&sh.x_full[xb]);
      for (int64_t c0 = 0; c0 < qchunks; c0 += a.pgroup) {
        const int cnt = int(qchunks - c0 < a.pgroup ? qchunks - c0 : a.pgroup);
        bool ok = true;
        if (ci < cnt) {
          uint32_t cs = cslot + uint32_t(ci), ph = cphase;
          if (cs >= nchunk) {
            cs -= nchunk;
            ph ^= 1u;
          }
          if (filled + uint64_t(ci) >= nchunk)
            ok = wait_phase(&sh.slot_empty[cs], ph ^ 1u, sh, a.status);
          const int64_t j = (c0 + ci) * CR + r;
          if (ok && j < a.N) {
            const uint64_t ell =
                sample_index(a.seed, uint64_t(q) * uint64_t(a.N) + uint64_t(j), uint64_t(a.L));
            if (a.ells_out) a.ells_out[q * a.N + j] = int64_t(ell);
            mbar_arrive_expect_tx(&sh.row_full[cs], a.row_bytes);
            bulk_g2s(ring + (size_t(cs) * CR + r) * a.row_bytes, R + int64_t(ell) * a.ldr,
                     a.row_bytes, &sh.row_full[cs]);
          } else if (ok) {
            mbar_arrive(&sh.row_full[cs]);  // past the end of the query: empty row
          }
        }
        if (__any_sync(0xffffffffu, !ok)) return;
        filled += uint64_t(cnt);
        cslot += uint32_t(cnt);
        if (cslot >= nchunk) {
          cslot -= nchunk;
          cphase ^= 1u;
        }
      }
    }
  } else if (warp < kFirstGatherWarp) {
    // ------------------------------------------------------------ coefficients
    const int cw = warp - kFirstCoefWarp;
    const int groups = int((a.n + 1023) / 1024);
    const uint32_t dmask = uint32_t(a.d - 1);
    uint32_t cs = uint32_t(cw), ph = 0;  // this warp handles chunks cw, cw + 3, ...
    uint64_t cc = uint64_t(cw);          // global chunk counter of this warp
    int qs = 0;
    float xr[32];
    for (int64_t q = blockIdx.x; q < a.Q; q += gridDim.x, ++qs) {
      const int xb = qs % kXBufs;
      if (!wait_phase(&sh.x_full[xb], uint32_t(qs / kXBufs) & 1u, sh, a.status)) return;
      const float* xq = xbuf + xb * a.xpad;
#pragma unroll
      for (int t = 0; t < 32; ++t) xr[t] = (XREG && t * 32 < a.xpad) ? xq[t * 32 + lane] : 0.f;
      const uint64_t cend = uint64_t(qs + 1) * uint64_t(qchunks);
      for (; cc < cend; cc += kCoefWarps) {
        const int64_t j0 = int64_t(cc - uint64_t(qs) * uint64_t(qchunks)) * CR;
        const int cnt = int(a.N - j0 < CR ? a.N - j0 : CR);
        // lanes 0..cnt-1 draw the chunk's indices; everyone gets all four
        uint32_t my_ell = 0;
        if (lane < cnt)
          my_ell = uint32_t(sample_index(
              a.seed, uint64_t(q) * uint64_t(a.N) + uint64_t(j0 + lane), uint64_t(a.L)));
        uint32_t ell[4];
#pragma unroll
        for (int s2 = 0; s2 < 4; ++s2) ell[s2] = __shfl_sync(0xffffffffu, my_ell, s2 < cnt ? s2 : 0);
        float c[4];
        kerdock_coefficients4<XREG>(a.tsigns, a.tsign_stride, ell, a.k, dmask, groups, lane, xr,
                                    xq, c);
        // the gather warps must be done with this chunk's previous samples
        if (cc >= nchunk && !wait_phase(&sh.slot_empty[cs], ph ^ 1u, sh, a.status)) return;
        if (lane == 0) {
#pragma unroll
          for (int s2 = 0; s2 < 4; ++s2) {
            if (s2 >= cnt) break;
            const uint32_t w = ell[s2] & dmask;
            float cv = c[s2];
            if (int64_t(ell[s2] >> a.k) == half) cv = w < a.n ? a.sqrt_d * xq[w] : 0.f;
            coef_s[cs * CR + s2] = cv;
            if (a.coef_out) a.coef_out[q * a.N + j0 + s2] = cv;
          }
          mbar_arrive(&sh.coef_full[cs]);
        }
        cs += kCoefWarps;
        if (cs >= nchunk) {
          cs -= nchunk;
          ph ^= 1u;
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&sh.x_empty[xb]);
    }
  } else if (warp < kFirstFinalWarp) {
    // ------------------------------------------------------------ gather
    const int gt = tid - kFirstGatherWarp * 32;
    uint32_t cs = 0, ph = 0;
    int qs = 0;
    for (int64_t q = blockIdx.x; q < a.Q; q += gridDim.x, ++qs) {
      const int mb = qs % kMBufs;
      float* means = means_base + int64_t(mb) * a.K * a.ldr;
      float acc[GPT][GR];
#pragma unroll
      for (int u = 0; u < GPT; ++u)
#pragma unroll
        for (int e = 0; e < GR; ++e) acc[u][e] = 0.f;
      int batch_left = a.J, batch = 0;
      for (int64_t j0 = 0; j0 < a.N; j0 += CR) {
        const int cnt = int(a.N - j0 < CR ? a.N - j0 : CR);
        if (!wait_phase(&sh.row_full[cs], ph, sh, a.status)) return;
        if (!wait_phase(&sh.coef_full[cs], ph, sh, a.status)) return;
#pragma unroll
        for (int s2 = 0; s2 < 4; ++s2) {
          if (s2 >= cnt) break;
          const float c = coef_s[cs * CR + s2];
          const unsigned char* row = ring + (size_t(cs) * CR + s2) * a.row_bytes;
#pragma unroll
          for (int u = 0; u < GPT; ++u) {
            const int gi = gt + u * kGatherThreads;
            if (gi * GR < a.ldr) {
              float v[GR];
              G::load(row + size_t(gi) * 16, v);
#pragma unroll
              for (int e = 0; e < GR; ++e) acc[u][e] = fmaf(c, v[e], acc[u][e]);
            }
          }
          if (--batch_left == 0) {
            if (batch == 0 && qs >= kMBufs &&
                !wait_phase(&sh.means_empty[mb], uint32_t(qs / kMBufs - 1) & 1u, sh, a.status))
              return;
            float* mrow = means + int64_t(batch) * a.ldr;
#pragma unroll
            for (int u = 0; u < GPT; ++u) {
              const int gi = gt + u * kGatherThreads;
              if (gi * GR < a.ldr) {
#pragma unroll
                for (int e = 0; e < GR; ++e) {
                  mrow[gi * GR + e] = acc[u][e] * a.inv_J;
                  acc[u][e] = 0.f;
                }
              }
            }
            batch_left = a.J;
            ++batch;
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&sh.slot_empty[cs]);
        if (++cs == nchunk) {
          cs = 0;
          ph ^= 1u;
        }
      }
      if (a.means_gmem != nullptr) __threadfence_block();
      __syncwarp();
      if (lane == 0) mbar_arrive(&sh.means_full[mb]);
    }
  } else {
    // ------------------------------------------------------------ finalizer
    const int ft = tid - kFirstFinalWarp * 32;
    const int fw = warp - kFirstFinalWarp;
    const int m = int(a.m);
    int qs = 0;
    for (int64_t q = blockIdx.x; q < a.Q; q += gridDim.x, ++qs) {
      const int mb = qs % kMBufs, xb = qs % kXBufs;
      if (!wait_phase(&sh.means_full[mb], uint32_t(qs / kMBufs) & 1u, sh, a.status)) return;
      if (!wait_phase(&sh.x_full[xb], uint32_t(qs / kXBufs) & 1u, sh, a.status)) return;
      const float* means = means_base + int64_t(mb) * a.K * a.ldr;
      const float* xq = xbuf + xb * a.xpad;
      // a6: median over the K batch means.
      for (int col = ft; col < m; col += kFinalThreads) {
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
        if (a.mu_out) a.mu_out[q * a.m + col] = med;
      }
      named_barrier_sync(kFinalBarrier, kFinalThreads);
      if (ft == 0) mbar_arrive(&sh.means_empty[mb]);  // means are consumed

      // a7: top-S by radix select on |mu| (4 digits of 8 bits, high first).
      uint32_t prefix = 0, mask = 0, remaining = uint32_t(a.S);
      for (int pass = 0; pass < 4; ++pass) {
        const int shift = 24 - 8 * pass;
        sh.hist[ft] = 0;
        sh.hist[ft + kFinalThreads] = 0;
        named_barrier_sync(kFinalBarrier, kFinalThreads);
        for (int i = ft; i < m; i += kFinalThreads) {
          const uint32_t key = abs_key(mus[i]);
          if ((key & mask) == prefix) atomicAdd(&sh.hist[(key >> shift) & 255u], 1u);
        }
        named_barrier_sync(kFinalBarrier, kFinalThreads);
        if (fw == 0) {
          const int base = (31 - lane) * 8;  // lane 0 holds the highest digits
          uint32_t sum = 0;
#pragma unroll
          for (int j2 = 0; j2 < 8; ++j2) sum += sh.hist[base + j2];
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
              const uint32_t h = sh.hist[base + j2];
              if (cum + h >= remaining) {
                sh.digit = uint32_t(base + j2);
                sh.remaining = remaining - cum;
                break;
              }
              cum += h;
            }
          }
        }
        named_barrier_sync(kFinalBarrier, kFinalThreads);
        prefix |= sh.digit << shift;
        mask |= 255u << shift;
        remaining = sh.remaining;
        named_barrier_sync(kFinalBarrier, kFinalThreads);
      }
      const uint32_t T = prefix;  // the S-th largest key; take `remaining` keys equal to T
      {
        const int seg = (m + kFinalThreads - 1) / kFinalThreads;
        const int lo = ft * seg, hi = lo + seg < m ? lo + seg : m;
        int eq = 0;
        for (int i = lo; i < hi; ++i) eq += abs_key(mus[i]) == T;
        int tot;
        int eq_rank = final_exclusive_scan(eq, sh.scan, &tot);
        const int eq_rank0 = eq_rank;
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
        int pos = final_exclusive_scan(take, sh.scan, &tot);
        eq_rank = eq_rank0;
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
      named_barrier_sync(kFinalBarrier, kFinalThreads);

      // a8: exact refinement v_i = a_i^T x, four rows per warp in flight.
      for (int r0 = fw * 4; r0 < a.S; r0 += kFinalWarps * 4) {
        float racc[4] = {0.f, 0.f, 0.f, 0.f};
        const float* arow[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
          arow[u] = a.A + int64_t(sel[r0 + u < a.S ? r0 + u : r0]) * a.lda;
        if (a.a_vec4) {
          const float4* xs4 = reinterpret_cast<const float4*>(xq);
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
            const float xv = xq[p];
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
      named_barrier_sync(kFinalBarrier, kFinalThreads);
      {
        const int seg = (a.S + kFinalThreads - 1) / kFinalThreads;
        const int lo = ft * seg, hi = lo + seg < a.S ? lo + seg : a.S;
        const bool full = a.flags & KERDOCK_FLAG_FULL_OUTPUT;
        int keep = 0;
        for (int r = lo; r < hi; ++r) keep += full || fabsf(vals[r]) >= a.eps;
        int tot;
        int pos = final_exclusive_scan(keep, sh.scan, &tot);
        const int64_t obase = q * a.S;
        for (int r = lo; r < hi; ++r) {
          if (full || fabsf(vals[r]) >= a.eps) {
            a.out_idx[obase + pos] = sel[r];
            a.out_val[obase + pos] = vals[r];
            ++pos;
          }
        }
        if (ft == 0) a.out_count[q] = tot;
      }
      named_barrier_sync(kFinalBarrier, kFinalThreads);
      if (ft == 0) mbar_arrive(&sh.x_empty[xb]);  // x of this query no longer needed
    }
  }
}

size_t align_up(size_t v, size_t al) { return (v + al - 1) / al * al; }

struct Layout {
  int nchunk, crows, pgroup;
  uint32_t row_bytes;
  size_t off_coef, off_x, off_means, off_mu, off_sel, off_vals, total;
  bool means_in_smem;
  int64_t xpad;
};

Layout make_layout(const Plan& p) {
  Layout L{};
  L.row_bytes = uint32_t(p.ldr * p.elem_bytes());
  L.xpad = p.d > 32 ? p.d : 32;
  const size_t spad = align_up(size_t(p.S), 4);
  const size_t means_bytes = size_t(kMBufs) * size_t(p.K) * size_t(p.ldr) * 4;
  L.means_in_smem = means_bytes <= kMeansSmemMax;
  // fixed (non-ring) parts, with slack for alignment
  const size_t fixed = size_t(kXBufs) * size_t(L.xpad) * 4 +
                       (L.means_in_smem ? means_bytes : 0) + size_t(p.ldr) * 4 +
                       2 * spad * 4 + 1024;
  const size_t per_slot = size_t(L.row_bytes) + 4;
  size_t avail = kSmemBudget > fixed ? kSmemBudget - fixed : 0;
  const size_t cap = kRingCap + size_t(kMaxSlots) * 4;
  if (avail > cap) avail = cap;
  int ns = int(avail / per_slot);
  if (ns > kMaxSlots) ns = kMaxSlots;
  // rows per chunk: four when the ring still holds at least 8 chunks
  L.crows = ns >= 32 ? 4 : ns >= 8 ? 2 : 1;
  L.nchunk = ns / L.crows;
  ns = L.nchunk * L.crows;
  int g = 1;  // chunks per producer step: g * crows <= 32 lanes, g <= nchunk / 2
  while (2 * g * L.crows <= 32 && 4 * g <= L.nchunk) g *= 2;
  L.pgroup = g;
  size_t off = align_up(size_t(ns) * L.row_bytes, 128);
  L.off_coef = off;
  off = align_up(off + size_t(ns) * 4, 16);
  L.off_x = off;
  off = align_up(off + size_t(kXBufs) * size_t(L.xpad) * 4, 16);
  L.off_means = off;
  if (L.means_in_smem) off = align_up(off + means_bytes, 16);
  L.off_mu = off;
  off = align_up(off + size_t(p.ldr) * 4, 16);
  L.off_sel = off;
  off = align_up(off + spad * 4, 16);
  L.off_vals = off;
  off = align_up(off + spad * 4, 16);
  L.total = off;
  return L;
}

template <typename RT, int GPT, bool XREG>
int launch_typed(const Plan& p, const Layout& L, QueryArgs& a, void* ws) {
  auto kern = query_kernel<RT, GPT, XREG>;
  KD_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   int(L.total)));
  int occ = 0;
  KD_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, L.total));
  if (occ < 1) return KERDOCK_ERR_UNSUPPORTED;
  int64_t grid = p.num_sms;
  if (grid > a.Q) grid = a.Q;
  a.means_gmem = L.means_in_smem ? nullptr : static_cast<float*>(ws);
  kern<<<unsigned(grid), kThreads, L.total, p.stream>>>(a);
  KD_CUDA_TRY(cudaGetLastError());
  return KERDOCK_OK;
}

}  // namespace

size_t apply_workspace_bytes(const Plan& p, int64_t q) {
  const Layout L = make_layout(p);
  if (L.means_in_smem || q == 0) return 0;
  const int64_t grid = p.num_sms > 0 ? p.num_sms : 256;
  return size_t(grid) * kMBufs * size_t(p.K) * size_t(p.ldr) * 4;
}

int launch_apply(const Plan& p, const float* X, int64_t q, int64_t ldx, float eps, uint64_t seed,
                 int flags, int32_t* out_idx, float* out_val, int32_t* out_count, void* ws,
                 size_t ws_bytes, float* mu_out, int64_t* ells_out, float* coef_out) {
  (void)ws_bytes;
  const Layout L = make_layout(p);
  if (L.nchunk < kMinChunks || L.total > kSmemBudget) return KERDOCK_ERR_UNSUPPORTED;
  QueryArgs a{};
  a.R = p.repr;
  a.tsigns = p.tsigns();
  a.tsign_stride = p.tsign_words;
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
  a.xpad = L.xpad;
  a.k = p.k;
  a.J = p.J;
  a.K = p.K;
  a.S = p.S;
  a.eps = eps;
  a.inv_J = 1.0f / float(p.J);
  a.sqrt_d = float(int64_t(1) << (p.k / 2));
  a.seed = seed;
  a.flags = flags;
  a.a_vec4 =
      (p.n % 4 == 0 && p.lda % 4 == 0 && (reinterpret_cast<uintptr_t>(p.A) & 15) == 0) ? 1 : 0;
  a.nchunk = L.nchunk;
  a.crows = L.crows;
  a.pgroup = L.pgroup;
  a.row_bytes = L.row_bytes;
  a.off_coef = uint32_t(L.off_coef);
  a.off_x = uint32_t(L.off_x);
  a.off_means = uint32_t(L.off_means);
  a.off_mu = uint32_t(L.off_mu);
  a.off_sel = uint32_t(L.off_sel);
  a.off_vals = uint32_t(L.off_vals);
  a.out_idx = out_idx;
  a.out_val = out_val;
  a.out_count = out_count;
  a.mu_out = mu_out;
  a.ells_out = ells_out;
  a.coef_out = coef_out;
  a.status = p.status();
  const int64_t granule = 16 / int64_t(p.elem_bytes());
  const int64_t gpt = (p.ldr / granule + kGatherThreads - 1) / kGatherThreads;
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

// ---------------------------------------------------------------------------
// Allocation-free apply.  Some callers cannot allocate device memory: code
// that runs while a stream is being captured into a CUDA graph, real-time or
// embedded hosts that fix their device-memory budget at start-up, or plugin
// hosts that own the allocator.  For them kerdock_apply_noalloc runs the same
// query kernel with its batch-mean scratch (normally the caller's workspace
// or shared memory) in this file-scope device array instead.  Every GPU that
// loads the library keeps the array until the process exits.  All calls share
// it, so calls that overlap on the GPU race with each other; nothing in it
// needs clearing, because each batch mean is written before it is read.
// ---------------------------------------------------------------------------
constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;  // 16 MiB
static __device__ __align__(256) float g_noalloc_scratch[kNoAllocScratchBytes / sizeof(float)];

namespace {

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (the host-side symbol is only a stand-in, never a device pointer).
int noalloc_scratch(void** out) {
  int dev = 0;
  KD_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices) return KERDOCK_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (g_noalloc_ptr[dev] == nullptr) {
    void* ptr = nullptr;
    KD_CUDA_TRY(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
    if (ptr == nullptr) return KERDOCK_ERR_CUDA;
    g_noalloc_ptr[dev] = ptr;
  }
  *out = g_noalloc_ptr[dev];
  return KERDOCK_OK;
}

// The kernel's shared-memory layout with the batch means always in global
// scratch (so the whole shared-memory budget goes to the row ring).
Layout make_layout_noalloc(const Plan& p) {
  Layout L{};
  L.row_bytes = uint32_t(p.ldr * p.elem_bytes());
  L.xpad = p.d > 32 ? p.d : 32;
  const size_t spad = align_up(size_t(p.S), 4);
  L.means_in_smem = false;
  const size_t fixed = size_t(kXBufs) * size_t(L.xpad) * 4 + size_t(p.ldr) * 4 + 2 * spad * 4 + 1024;
  const size_t per_slot = size_t(L.row_bytes) + 4;
  size_t avail = kSmemBudget > fixed ? kSmemBudget - fixed : 0;
  const size_t cap = kRingCap + size_t(kMaxSlots) * 4;
  if (avail > cap) avail = cap;
  int ns = int(avail / per_slot);
  if (ns > kMaxSlots) ns = kMaxSlots;
  L.crows = ns >= 32 ? 4 : ns >= 8 ? 2 : 1;
  L.nchunk = ns / L.crows;
  ns = L.nchunk * L.crows;
  int g = 1;
  while (2 * g * L.crows <= 32 && 4 * g <= L.nchunk) g *= 2;
  L.pgroup = g;
  size_t off = align_up(size_t(ns) * L.row_bytes, 128);
  L.off_coef = off;
  off = align_up(off + size_t(ns) * 4, 16);
  L.off_x = off;
  off = align_up(off + size_t(kXBufs) * size_t(L.xpad) * 4, 16);
  L.off_means = off;
  L.off_mu = off;
  off = align_up(off + size_t(p.ldr) * 4, 16);
  L.off_sel = off;
  off = align_up(off + spad * 4, 16);
  L.off_vals = off;
  off = align_up(off + spad * 4, 16);
  L.total = off;
  return L;
}

template <typename RT, int GPT, bool XREG>
int launch_noalloc_typed(const Layout& L, QueryArgs& a, int64_t grid, cudaStream_t stream) {
  auto kern = query_kernel<RT, GPT, XREG>;
  KD_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   int(L.total)));
  kern<<<unsigned(grid), kThreads, L.total, stream>>>(a);
  KD_CUDA_TRY(cudaGetLastError());
  return KERDOCK_OK;
}

}  // namespace

size_t noalloc_scratch_bytes() { return kNoAllocScratchBytes; }

int launch_apply_noalloc(const Plan& p, const float* X, int64_t q, int64_t ldx, float eps,
                         uint64_t seed, int flags, int32_t* out_idx, float* out_val,
                         int32_t* out_count) {
  const Layout L = make_layout_noalloc(p);
  if (L.nchunk < kMinChunks || L.total > kSmemBudget) return KERDOCK_ERR_UNSUPPORTED;
  int64_t grid = p.num_sms;
  if (grid > q) grid = q;
  const size_t need = size_t(grid) * kMBufs * size_t(p.K) * size_t(p.ldr) * sizeof(float);
  if (need > kNoAllocScratchBytes) return KERDOCK_ERR_CAPACITY;  // beyond the fixed scratch
  void* scratch = nullptr;
  const int rc = noalloc_scratch(&scratch);
  if (rc != KERDOCK_OK) return rc;
  QueryArgs a{};
  a.R = p.repr;
  a.tsigns = p.tsigns();
  a.tsign_stride = p.tsign_words;
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
  a.xpad = L.xpad;
  a.k = p.k;
  a.J = p.J;
  a.K = p.K;
  a.S = p.S;
  a.eps = eps;
  a.inv_J = 1.0f / float(p.J);
  a.sqrt_d = float(int64_t(1) << (p.k / 2));
  a.seed = seed;
  a.flags = flags;
  a.a_vec4 =
      (p.n % 4 == 0 && p.lda % 4 == 0 && (reinterpret_cast<uintptr_t>(p.A) & 15) == 0) ? 1 : 0;
  a.nchunk = L.nchunk;
  a.crows = L.crows;
  a.pgroup = L.pgroup;
  a.row_bytes = L.row_bytes;
  a.off_coef = uint32_t(L.off_coef);
  a.off_x = uint32_t(L.off_x);
  a.off_means = uint32_t(L.off_means);
  a.off_mu = uint32_t(L.off_mu);
  a.off_sel = uint32_t(L.off_sel);
  a.off_vals = uint32_t(L.off_vals);
  a.means_gmem = static_cast<float*>(scratch);
  a.out_idx = out_idx;
  a.out_val = out_val;
  a.out_count = out_count;
  a.status = p.status();
  const int64_t granule = 16 / int64_t(p.elem_bytes());
  const int64_t gpt = (p.ldr / granule + kGatherThreads - 1) / kGatherThreads;
  const bool xreg = p.n <= 1024;
  if (p.dtype == KERDOCK_BF16) {
    if (gpt <= 1) return xreg ? launch_noalloc_typed<__nv_bfloat16, 1, true>(L, a, grid, p.stream)
                              : launch_noalloc_typed<__nv_bfloat16, 1, false>(L, a, grid, p.stream);
    if (gpt <= 2) return xreg ? launch_noalloc_typed<__nv_bfloat16, 2, true>(L, a, grid, p.stream)
                              : launch_noalloc_typed<__nv_bfloat16, 2, false>(L, a, grid, p.stream);
    return launch_noalloc_typed<__nv_bfloat16, 4, false>(L, a, grid, p.stream);
  }
  if (gpt <= 1) return xreg ? launch_noalloc_typed<float, 1, true>(L, a, grid, p.stream)
                            : launch_noalloc_typed<float, 1, false>(L, a, grid, p.stream);
  if (gpt <= 2) return xreg ? launch_noalloc_typed<float, 2, true>(L, a, grid, p.stream)
                            : launch_noalloc_typed<float, 2, false>(L, a, grid, p.stream);
  return launch_noalloc_typed<float, 4, false>(L, a, grid, p.stream);
}

}  // namespace kd
