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
//                 c_j for a ring chunk's samples (1, 2 or 4) at a time from
//                 the lane-transposed sign table and x, ahead of the gather.
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
#include <type_traits>

#include "kerdock_internal.cuh"

namespace kd {
namespace {

// Warp roles: warp 0 produces, warps [1, 1 + CW) compute coefficients,
// warps [1 + CW, 12) gather and warps [12, 16) finalize.  A coefficient costs n
// sign-adds and a gathered row m multiply-adds, so the best split follows n/m:
// measured on GB300 with m = n = 4096 (bfloat16), CW = 3 took 17.3 ms for 4096
// queries against 19.3 ms (CW = 4) and 20.0 ms (CW = 5), while with m = 256,
// n = 4096 CW = 5 was 1.7x faster than CW = 3.  At m = n = 1024 a float32 row
// is cheap to gather per byte and the coefficients set the pace: CW = 5 took
// 0.573 ms for 1000 queries against 0.578 (CW = 4) and 0.631 ms (CW = 3); a
// bfloat16 row costs the gather warps an unpacking step per element, and there
// CW = 3 is best (0.655 ms against 0.696 and 0.687, and 0.841 ms with CW = 2;
// at n = 4096, CW = 2 took 22.3 ms against 17.3 ms).
constexpr int kFinalWarps = 4;
constexpr int kFirstCoefWarp = 1;
constexpr int kWarps = 16;
constexpr int kFirstFinalWarp = kWarps - kFinalWarps;
constexpr int kThreads = kWarps * 32;                   // 512
constexpr int kFinalThreads = kFinalWarps * 32;
constexpr int kCoefWarpsSmallF32 = 5;   // n <= 1024, float32 rows
constexpr int kCoefWarpsSmallBf16 = 3;  // n <= 1024, bfloat16 rows
constexpr int kCoefWarpsLarge = 3;      // n > 1024, float32 rows
constexpr int kCoefWarpsLargeBf16 = 3;  // n > 1024, bfloat16 rows
constexpr int kCoefWarpsBatch = 3;      // mixed plans
// the split of a single-plan kernel
template <typename RT, bool XREG>
constexpr int coef_warps() {
  return sizeof(RT) == 2 ? (XREG ? kCoefWarpsSmallBf16 : kCoefWarpsLargeBf16)
                         : (XREG ? kCoefWarpsSmallF32 : kCoefWarpsLarge);
}
template <int CW>
struct Roles {
  static constexpr int kCoefWarps = CW;
  static constexpr int kFirstGatherWarp = kFirstCoefWarp + CW;
  static constexpr int kGatherWarps = kFirstFinalWarp - kFirstGatherWarp;
  static constexpr int kGatherThreads = kGatherWarps * 32;
};
constexpr int kMaxSlots = 128;  // ring slots
constexpr int kMaxChunkRows = 32;  // rows of one packed chunk: one producer lane each
constexpr int kMaxChunks = 64;
// > every CW: each coefficient warp steps CW chunks and starts at chunk cw < CW
// The ring must hold more chunks than the kernel's coefficient warps: each
// coefficient warp steps CW chunks and starts at chunk cw < CW (Dims::coef_warps).
static_assert(Dims{}.coef_warps == kCoefWarpsBatch, "the batch kernel's split is the default");
constexpr int kXBufs = 3;
constexpr int kMBufs = 2;
constexpr int kFinalBarrier = 1;  // named barrier id of the finalizer warps
constexpr size_t kSmemBudget = 227 * 1024 - 4096;  // dynamic bytes (static ~3 KB)
constexpr size_t kRingCap = 160 * 1024;
constexpr size_t kMeansSmemMax = 32 * 1024;  // larger batch means go to global memory, leaving the ring its space

// acc = c * v + acc on two float lanes at once (fma.rn.f32x2: each lane is the
// same single-rounding FMA as fmaf).
__device__ __forceinline__ float2 fma2(float2 c, float2 v, float2 acc) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;"
      : "=l"(r)
      : "l"(*reinterpret_cast<unsigned long long*>(&c)),
        "l"(*reinterpret_cast<unsigned long long*>(&v)),
        "l"(*reinterpret_cast<unsigned long long*>(&acc)));
  return *reinterpret_cast<float2*>(&r);
}

// One 16-byte granule of a representation row: acc[e] += c * (elements 2e, 2e+1).
template <typename RT>
struct Granule;
template <>
struct Granule<float> {
  static constexpr int kElems = 4;
  __device__ static void fma(const unsigned char* p, float2 c2, float2 (&acc)[2]) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    acc[0] = fma2(c2, make_float2(v.x, v.y), acc[0]);
    acc[1] = fma2(c2, make_float2(v.z, v.w), acc[1]);
  }
};
template <>
struct Granule<__nv_bfloat16> {
  static constexpr int kElems = 8;
  // a bfloat16 is the top half of the float32 with the same value
  __device__ static void fma(const unsigned char* p, float2 c2, float2 (&acc)[4]) {
    const uint4 v = *reinterpret_cast<const uint4*>(p);
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int e = 0; e < 4; ++e)
      acc[e] = fma2(c2, make_float2(__uint_as_float(w[e] << 16), __uint_as_float(w[e] & 0xffff0000u)),
                    acc[e]);
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
template <bool XREG, int NS>
__device__ __forceinline__ void kerdock_coefficients(const uint32_t* __restrict__ tsigns,
                                                     int64_t tstride, const uint32_t (&ell)[4],
                                                     int kbits, uint32_t dmask, int groups,
                                                     int lane, const float (&xr)[32],
                                                     const float* xs, float (&c)[4]) {
  // d <= 4096: at most four 1024-point groups; x in registers means n <= 1024
  constexpr int kMaxGroups = XREG ? 1 : 4;
  float part[NS];
  uint32_t whi[NS], pl[NS], wmask[NS];
  const uint32_t* rows[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    part[s] = 0.f;
    const uint32_t w = ell[s] & dmask;
    whi[s] = w >> 5;
    pl[s] = __popc(w & 31u & uint32_t(lane)) & 1u;
    wmask[s] = __ballot_sync(0xffffffffu, __popc(whi[s] & 31u & uint32_t(lane)) & 1u);
    // identity-basis samples (b = d/2) read row d/2 - 1; their result is replaced
    const uint32_t b = ell[s] >> kbits;
    const uint32_t bmax = (dmask + 1u) / 2u - 1u;
    rows[s] = tsigns + int64_t(b < bmax ? b : bmax) * tstride;
  }
  // every group's sign words are requested before the first is used
  uint32_t F[kMaxGroups][NS];
#pragma unroll
  for (int g = 0; g < kMaxGroups; ++g)
#pragma unroll
    for (int s = 0; s < NS; ++s) F[g][s] = g < groups ? __ldg(rows[s] + (g << 5) + lane) : 0u;
#pragma unroll
  for (int g = 0; g < kMaxGroups; ++g) {
    if (g >= groups) break;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      F[g][s] ^= wmask[s];
      if ((__popc(whi[s] & uint32_t(g << 5)) & 1u) ^ pl[s]) F[g][s] = ~F[g][s];
    }
#pragma unroll
    for (int t = 0; t < 32; ++t) {
      const float xv = XREG ? xr[t] : xs[((g << 5) + t) * 32 + lane];
#pragma unroll
      for (int s = 0; s < NS; ++s)
        part[s] += __uint_as_float(__float_as_uint(xv) ^ ((F[g][s] << (31 - t)) & 0x80000000u));
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int s = 0; s < NS; ++s) part[s] += __shfl_xor_sync(0xffffffffu, part[s], o);
#pragma unroll
  for (int s = 0; s < 4; ++s) c[s] = s < NS ? part[s] : 0.f;
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
  int abort_flag;       // a wait ran out: every role stops
  int final_abort;      // the finalizer warps' shared decision to stop
  uint32_t armed[kMaxChunks];  // 1 + global fill number of each chunk's last arming (0: never)
};

// Bounded wait that also gives up once another role has aborted.  After
// cfg.poll_limit unsuccessful polls it records a timeout in the status word
// and raises the CTA's abort flag.
__device__ __forceinline__ bool wait_phase(uint64_t* bar, uint32_t parity, Shared& sh,
                                           const LaunchCfg& cfg) {
  for (uint32_t it = 0;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    const bool limit = it >= cfg.poll_limit;
    if ((it & 255u) == 255u || limit) {
      if (*reinterpret_cast<volatile int*>(&sh.abort_flag)) return false;
      if (limit) {
        set_status(cfg.status, kStatusTimeout);
        *reinterpret_cast<volatile int*>(&sh.abort_flag) = 1;
        return false;
      }
    }
  }
}

// A wait whose outcome the whole warp shares: if any lane gave up, every lane
// returns false, so a warp never splits between stopping and going on to its
// next warp-wide instruction.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, Shared& sh,
                                          const LaunchCfg& cfg) {
  return __all_sync(0xffffffffu, wait_phase(bar, parity, sh, cfg));
}

// Single-plan launch: the plan-wide descriptor plus the query batch shape.
struct QueryArgs {
  LaunchCfg cfg;
  QueryDesc base;  // x, outputs and debug pointers point at query 0
  int64_t Q, ldx;
};

// Batch launch: descriptors, their order and each CTA's range in it.
struct BatchArgs {
  LaunchCfg cfg;
  const QueryDesc* descs;
  const int32_t* order;
  const int64_t* cta_start;  // gridDim.x + 1 entries
};

struct SingleSeq {
  const QueryArgs& a;
  __device__ int64_t size() const {
    return blockIdx.x < a.Q ? (a.Q - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  }
  __device__ QueryDesc get(int64_t i) const {
    const int64_t q = blockIdx.x + i * gridDim.x;
    QueryDesc d = a.base;
    d.x = a.base.x + q * a.ldx;
    d.out_idx = a.base.out_idx + q * a.base.S;
    d.out_val = a.base.out_val + q * a.base.S;
    d.out_count = a.base.out_count + q;
    if (d.mu_out) d.mu_out += q * a.base.m;
    if (d.ells_out) d.ells_out += q * a.base.N;
    if (d.coef_out) d.coef_out += q * a.base.N;
    d.ctr_base = q * a.base.N;
    return d;
  }
};

struct BatchSeq {
  const BatchArgs& a;
  __device__ int64_t size() const { return a.cta_start[blockIdx.x + 1] - a.cta_start[blockIdx.x]; }
  __device__ QueryDesc get(int64_t i) const { return a.descs[a.order[a.cta_start[blockIdx.x] + i]]; }
};

// Shared-memory regions of a launch.
struct Regions {
  unsigned char* ring;
  float* coef_s;
  float* xbuf;
  float* means_base;
  float* mus;
  int32_t* sel;
  float* vals;
};

__device__ __forceinline__ Regions regions(unsigned char* smem, const LaunchCfg& c) {
  Regions r;
  r.ring = smem;
  r.coef_s = reinterpret_cast<float*>(smem + c.off_coef);
  r.xbuf = reinterpret_cast<float*>(smem + c.off_x);
  r.means_base = c.means_gmem != nullptr ? c.means_gmem + int64_t(blockIdx.x) * kMBufs * c.mstride
                                         : reinterpret_cast<float*>(smem + c.off_means);
  r.mus = reinterpret_cast<float*>(smem + c.off_mu);
  r.sel = reinterpret_cast<int32_t*>(smem + c.off_sel);
  r.vals = reinterpret_cast<float*>(smem + c.off_vals);
  return r;
}

template <int CW>
__device__ __forceinline__ void init_barriers(Shared& sh, const LaunchCfg& c) {
  using RL = Roles<CW>;
  if (threadIdx.x == 0) {
    for (int s = 0; s < c.nchunk; ++s) {
      mbar_init(&sh.row_full[s], uint32_t(c.crows));
      mbar_init(&sh.coef_full[s], 1);
      mbar_init(&sh.slot_empty[s], RL::kGatherWarps);
    }
    for (int b = 0; b < kXBufs; ++b) {
      mbar_init(&sh.x_full[b], 1);
      mbar_init(&sh.x_empty[b], RL::kCoefWarps + 1);
    }
    for (int b = 0; b < kMBufs; ++b) {
      mbar_init(&sh.means_full[b], RL::kGatherWarps);
      mbar_init(&sh.means_empty[b], 1);
    }
    sh.abort_flag = 0;
    sh.final_abort = 0;
    for (int s = 0; s < kMaxChunks; ++s) sh.armed[s] = 0;
    fence_mbar_init();
  }
  __syncthreads();
}

// Rows of a query per ring slot in a batch launch.  A batch's slot is as large
// as its largest row; a query whose rows are at most half of it packs 2, 4,
// ... rows into each slot (a chunk then carries crows * rows_per_slot
// consecutive samples, at most kMaxChunkRows), so the small rows of a mixed
// batch keep more bytes in flight and pay a chunk's barriers once per several
// rows.  Single-plan launches keep one row per slot (the slot is the row),
// and their code is compiled without the packed paths.
__device__ __forceinline__ int rows_per_slot(const QueryDesc& qd, const LaunchCfg& cfg) {
  int rps = 1;
  while (2u * uint32_t(rps) * qd.row_bytes <= cfg.slot_bytes &&
         2 * rps * cfg.crows <= kMaxChunkRows)
    rps *= 2;
  return rps;
}

// ---------------------------------------------------------------- producer
template <class Seq>
__device__ void producer_role(const Seq& seq, const LaunchCfg& cfg, const Regions& rg, Shared& sh) {
  constexpr bool kPack = std::is_same<Seq, BatchSeq>::value;
  const int lane = threadIdx.x & 31;
  const int CR = cfg.crows;
  const uint32_t nchunk = uint32_t(cfg.nchunk);
  uint32_t cslot = 0, cphase = 0;  // ring chunk of the next chunk to fill and its phase
  uint64_t filled = 0;             // chunks filled so far
  const int64_t nq = seq.size();
  for (int64_t qs = 0; qs < nq; ++qs) {
    const QueryDesc qd = seq.get(qs);
    const int xb = int(qs % kXBufs);
    if (qs >= kXBufs && !warp_wait(&sh.x_empty[xb], uint32_t(qs / kXBufs - 1) & 1u, sh, cfg))
      return;
    float* xq = rg.xbuf + xb * cfg.xpad;
    for (int64_t p = lane; p < cfg.xpad; p += 32) xq[p] = p < qd.n ? qd.x[p] : 0.f;
    __syncwarp();
    if (lane == 0) mbar_arrive(&sh.x_full[xb]);
    // RPC rows per chunk (a power of two), one lane each; pg chunks per step
    const int rps = kPack ? rows_per_slot(qd, cfg) : 1, RPC = CR * rps;
    const int pg = cfg.pgroup < 32 / RPC ? cfg.pgroup : 32 / RPC;
    const int ci = lane / RPC, r = lane % RPC;
    // the RPC lanes that fill one chunk
    const uint32_t chunk_mask = RPC == 32 ? 0xffffffffu : ((1u << RPC) - 1u) << (ci * RPC);
    const int64_t qchunks = (qd.N + RPC - 1) / RPC;
    const unsigned char* R = static_cast<const unsigned char*>(qd.R);
    for (int64_t c0 = 0; c0 < qchunks; c0 += pg) {
      const int cnt = int(qchunks - c0 < pg ? qchunks - c0 : pg);
      bool ok = true;
      uint32_t cs = cslot + uint32_t(ci), ph = cphase;
      if (cs >= nchunk) {
        cs -= nchunk;
        ph ^= 1u;
      }
      if (ci < cnt && filled + uint64_t(ci) >= nchunk)
        ok = wait_phase(&sh.slot_empty[cs], ph ^ 1u, sh, cfg);
      // the lanes of one chunk arm it together or not at all, so an abort
      // leaves no chunk partly armed; each armed chunk records its fill number
      ok = __all_sync(chunk_mask, ok);
      // Row r of a chunk goes to byte r * row_bytes of the chunk's CR slots.
      // With one row per slot each lane arrives with its own bytes; with
      // packed slots every copy's bytes are expected before any arrival and
      // the first lane of each slot arrives once (a slot past the end of the
      // query arrives empty), so the CR arrivals close the phase only when
      // every row has landed.
      if (ci < cnt && ok) {
        if (r == 0) sh.armed[cs] = uint32_t(filled + uint64_t(ci) + 1);
        const int64_t j = (c0 + ci) * RPC + r;
        if (j < qd.N) {
          const uint64_t ell =
              sample_index(qd.seed, uint64_t(qd.ctr_base) + uint64_t(j), uint64_t(qd.L));
          if (qd.ells_out) qd.ells_out[j] = int64_t(ell);
          if (rps == 1)
            mbar_arrive_expect_tx(&sh.row_full[cs], qd.row_bytes);
          else
            mbar_expect_tx(&sh.row_full[cs], qd.row_bytes);
          bulk_g2s(rg.ring + size_t(cs) * CR * cfg.slot_bytes + size_t(r) * qd.row_bytes,
                   R + int64_t(ell) * qd.row_bytes, qd.row_bytes, &sh.row_full[cs]);
        } else if (rps == 1) {
          mbar_arrive(&sh.row_full[cs]);  // past the end of the query: empty row
        }
      }
      if (kPack && rps > 1) {
        __syncwarp();
        if (ci < cnt && ok && r % rps == 0) mbar_arrive(&sh.row_full[cs]);
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
}

// ---------------------------------------------------------------- coefficients
struct CoefState {
  uint32_t cs, ph;  // ring chunk and phase of this warp's next chunk
  uint64_t cc;      // global chunk counter of this warp's next chunk
  uint64_t cbase;   // global chunk counter of the current query's first chunk
};


// kerdock_coefficients in two halves, so that a coefficient warp can request
// the sign words of its next chunk (coef_issue) before it sums the current one
// (coef_finish): the words' load latency then overlaps the sums.
template <bool XREG, int NS>
struct CoefWords {
  static constexpr int kMaxGroups = XREG ? 1 : 4;
  uint32_t F[kMaxGroups][NS];
};
template <bool XREG, int NS>
__device__ __forceinline__ void coef_issue(const uint32_t* __restrict__ tsigns, int64_t tstride,
                                           const uint32_t (&ell)[4], int kbits, uint32_t dmask,
                                           int groups, int lane, CoefWords<XREG, NS>& W) {
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    const uint32_t b = ell[s] >> kbits;
    const uint32_t bmax = (dmask + 1u) / 2u - 1u;
    const uint32_t* row = tsigns + int64_t(b < bmax ? b : bmax) * tstride;
#pragma unroll
    for (int g = 0; g < CoefWords<XREG, NS>::kMaxGroups; ++g)
      W.F[g][s] = g < groups ? __ldg(row + (g << 5) + lane) : 0u;
  }
}
template <bool XREG, int NS>
__device__ __forceinline__ void coef_finish(CoefWords<XREG, NS>& W, const uint32_t (&ell)[4],
                                            uint32_t dmask, int groups, int lane,
                                            const float (&xr)[32], const float* xs, float (&c)[4]) {
  constexpr int kMaxGroups = CoefWords<XREG, NS>::kMaxGroups;
  float part[NS];
  uint32_t whi[NS], pl[NS], wmask[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    part[s] = 0.f;
    const uint32_t w = ell[s] & dmask;
    whi[s] = w >> 5;
    pl[s] = __popc(w & 31u & uint32_t(lane)) & 1u;
    wmask[s] = __ballot_sync(0xffffffffu, __popc(whi[s] & 31u & uint32_t(lane)) & 1u);
  }
#pragma unroll
  for (int g = 0; g < kMaxGroups; ++g) {
    if (g >= groups) break;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      W.F[g][s] ^= wmask[s];
      if ((__popc(whi[s] & uint32_t(g << 5)) & 1u) ^ pl[s]) W.F[g][s] = ~W.F[g][s];
    }
#pragma unroll
    for (int t = 0; t < 32; ++t) {
      const float xv = XREG ? xr[t] : xs[((g << 5) + t) * 32 + lane];
#pragma unroll
      for (int s = 0; s < NS; ++s)
        part[s] += __uint_as_float(__float_as_uint(xv) ^ ((W.F[g][s] << (31 - t)) & 0x80000000u));
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int s = 0; s < NS; ++s) part[s] += __shfl_xor_sync(0xffffffffu, part[s], o);
#pragma unroll
  for (int s = 0; s < 4; ++s) c[s] = s < NS ? part[s] : 0.f;
}

// One query's chunks for this coefficient warp (every CW-th chunk, NS rows
// each), with the next chunk's samples drawn and its sign words requested
// before the current chunk is summed.  Used by the single-plan kernels with x
// in registers (n <= 1024) and chunks of up to four rows: 3 % less time for
// the n = 1024 float32 queries (0.644 against 0.662 ms for 1000); with x in
// shared memory the second set of words spills registers.
template <bool XREG, int NS, int CW>
__device__ bool coef_chunks_pf(const QueryDesc& qd, CoefState& st, const LaunchCfg& cfg,
                               const Regions& rg, Shared& sh, const float* xq,
                               const float (&xr)[32], uint64_t cend) {
  const int lane = threadIdx.x & 31;
  const uint32_t nchunk = uint32_t(cfg.nchunk);
  const int groups = int((qd.n + 1023) / 1024);
  const uint32_t dmask = uint32_t(qd.d - 1);
  const int64_t half = qd.d / 2;
  auto draw = [&](uint64_t cc, uint32_t (&ell)[4]) {
    const int64_t j0 = int64_t(cc - st.cbase) * NS;
    const int cnt = int(qd.N - j0 < NS ? qd.N - j0 : NS);
    uint32_t my_ell = 0;
    if (lane < cnt)
      my_ell = uint32_t(
          sample_index(qd.seed, uint64_t(qd.ctr_base) + uint64_t(j0 + lane), uint64_t(qd.L)));
#pragma unroll
    for (int s2 = 0; s2 < 4; ++s2) ell[s2] = __shfl_sync(0xffffffffu, my_ell, s2 < cnt ? s2 : 0);
  };
  uint32_t ell[4];
  CoefWords<XREG, NS> W;
  if (st.cc < cend) {
    draw(st.cc, ell);
    coef_issue<XREG, NS>(qd.tsigns, qd.tstride, ell, qd.k, dmask, groups, lane, W);
  }
  for (; st.cc < cend; st.cc += CW) {
    const int64_t j0 = int64_t(st.cc - st.cbase) * NS;
    const int cnt = int(qd.N - j0 < NS ? qd.N - j0 : NS);
    uint32_t ell_next[4] = {0u, 0u, 0u, 0u};
    CoefWords<XREG, NS> Wn;
    if (st.cc + CW < cend) {
      draw(st.cc + CW, ell_next);
      coef_issue<XREG, NS>(qd.tsigns, qd.tstride, ell_next, qd.k, dmask, groups, lane, Wn);
    }
    float c[4];
    coef_finish<XREG, NS>(W, ell, dmask, groups, lane, xr, xq, c);
    if (st.cc >= nchunk && !warp_wait(&sh.slot_empty[st.cs], st.ph ^ 1u, sh, cfg)) return false;
    if (lane == 0) {
#pragma unroll
      for (int s2 = 0; s2 < 4; ++s2) {
        if (s2 >= cnt) break;
        const uint32_t w = ell[s2] & dmask;
        float cv = c[s2];
        if (int64_t(ell[s2] >> qd.k) == half) cv = w < qd.n ? qd.sqrt_d * xq[w] : 0.f;
        rg.coef_s[st.cs * NS + s2] = cv;
        if (qd.coef_out) qd.coef_out[j0 + s2] = cv;
      }
      mbar_arrive(&sh.coef_full[st.cs]);
    }
    st.cs += CW;
    if (st.cs >= nchunk) {
      st.cs -= nchunk;
      st.ph ^= 1u;
    }
#pragma unroll
    for (int s2 = 0; s2 < 4; ++s2) ell[s2] = ell_next[s2];
    W = Wn;
  }
  return true;
}

// PACK (the batch kernel): a chunk holds crows * rows_per_slot samples, up to
// kMaxChunkRows, computed four at a time with each lane keeping its own
// sample's coefficient; the coefficient area has kMaxChunkRows entries per
// chunk.
template <bool XREG, int CW, bool PACK>
__device__ bool coef_query(const QueryDesc& qd, int64_t qs, CoefState& st, const LaunchCfg& cfg,
                           const Regions& rg, Shared& sh, const float* xq) {
  const int lane = threadIdx.x & 31;
  const int CR = cfg.crows;
  const uint32_t nchunk = uint32_t(cfg.nchunk);
  const int groups = int((qd.n + 1023) / 1024);
  const uint32_t dmask = uint32_t(qd.d - 1);
  const int64_t half = qd.d / 2;
  float xr[32];
#pragma unroll
  for (int t = 0; t < 32; ++t) xr[t] = (XREG && t * 32 < cfg.xpad) ? xq[t * 32 + lane] : 0.f;
  if constexpr (PACK) {
    const int RPC = CR * rows_per_slot(qd, cfg);
    const uint64_t cend = st.cbase + uint64_t((qd.N + RPC - 1) / RPC);
    for (; st.cc < cend; st.cc += CW) {
      const int64_t j0 = int64_t(st.cc - st.cbase) * RPC;
      const int cnt = int(qd.N - j0 < RPC ? qd.N - j0 : RPC);
      // lane s draws sample j0 + s of the chunk and keeps its coefficient
      uint32_t my_ell = 0;
      if (lane < cnt)
        my_ell = uint32_t(
            sample_index(qd.seed, uint64_t(qd.ctr_base) + uint64_t(j0 + lane), uint64_t(qd.L)));
      float my_c = 0.f;
      for (int h = 0; h < cnt; h += 4) {
        uint32_t ell[4];
#pragma unroll
        for (int s2 = 0; s2 < 4; ++s2)
          ell[s2] = __shfl_sync(0xffffffffu, my_ell, h + s2 < cnt ? h + s2 : h);
        float c[4];
        if (RPC >= 4)
          kerdock_coefficients<XREG, 4>(qd.tsigns, qd.tstride, ell, qd.k, dmask, groups, lane, xr,
                                        xq, c);
        else if (RPC == 2)
          kerdock_coefficients<XREG, 2>(qd.tsigns, qd.tstride, ell, qd.k, dmask, groups, lane, xr,
                                        xq, c);
        else
          kerdock_coefficients<XREG, 1>(qd.tsigns, qd.tstride, ell, qd.k, dmask, groups, lane, xr,
                                        xq, c);
#pragma unroll
        for (int s2 = 0; s2 < 4; ++s2)
          if (lane == h + s2) my_c = c[s2];
      }
      // the gather warps must be done with this chunk's previous samples
      if (st.cc >= nchunk && !warp_wait(&sh.slot_empty[st.cs], st.ph ^ 1u, sh, cfg)) return false;
      if (lane < cnt) {
        const uint32_t w = my_ell & dmask;
        if (int64_t(my_ell >> qd.k) == half) my_c = w < qd.n ? qd.sqrt_d * xq[w] : 0.f;
        rg.coef_s[st.cs * kMaxChunkRows + lane] = my_c;
        if (qd.coef_out) qd.coef_out[j0 + lane] = my_c;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&sh.coef_full[st.cs]);
      st.cs += CW;
      if (st.cs >= nchunk) {
        st.cs -= nchunk;
        st.ph ^= 1u;
      }
    }
    st.cbase = cend;
    return true;
  }
  const uint64_t cend = st.cbase + uint64_t((qd.N + CR - 1) / CR);
  if (XREG && CR <= 4) {  // the pipelined form (coef_chunks_pf)
    bool ok;
    if (CR == 4) ok = coef_chunks_pf<XREG, 4, CW>(qd, st, cfg, rg, sh, xq, xr, cend);
    else if (CR == 2) ok = coef_chunks_pf<XREG, 2, CW>(qd, st, cfg, rg, sh, xq, xr, cend);
    else ok = coef_chunks_pf<XREG, 1, CW>(qd, st, cfg, rg, sh, xq, xr, cend);
    if (!ok) return false;
    st.cbase = cend;
    return true;
  }
  for (; st.cc < cend; st.cc += CW) {
    const int64_t j0 = int64_t(st.cc - st.cbase) * CR;
    const int cnt = int(qd.N - j0 < CR ? qd.N - j0 : CR);
    // lanes 0..cnt-1 draw the chunk's indices; every lane gets all of them
    uint32_t my_ell = 0;
    if (lane < cnt)
      my_ell = uint32_t(
          sample_index(qd.seed, uint64_t(qd.ctr_base) + uint64_t(j0 + lane), uint64_t(qd.L)));
    uint32_t ell[8];
#pragma unroll
    for (int s2 = 0; s2 < 8; ++s2) ell[s2] = __shfl_sync(0xffffffffu, my_ell, s2 < cnt ? s2 : 0);
    float c[8];
    // a chunk holds CR samples: compute exactly those (CR is uniform per
    // launch), four at a time
    if (CR >= 4) {
      const uint32_t e0[4] = {ell[0], ell[1], ell[2], ell[3]};
      float c0[4];
      kerdock_coefficients<XREG, 4>(qd.tsigns, qd.tstride, e0, qd.k, dmask, groups, lane, xr, xq, c0);
#pragma unroll
      for (int s2 = 0; s2 < 4; ++s2) c[s2] = c0[s2];
      if (CR == 8) {
        const uint32_t e1[4] = {ell[4], ell[5], ell[6], ell[7]};
        kerdock_coefficients<XREG, 4>(qd.tsigns, qd.tstride, e1, qd.k, dmask, groups, lane, xr, xq,
                                      c0);
#pragma unroll
        for (int s2 = 0; s2 < 4; ++s2) c[4 + s2] = c0[s2];
      }
    } else {
      const uint32_t e0[4] = {ell[0], ell[1], ell[2], ell[3]};
      float c0[4];
      if (CR == 2)
        kerdock_coefficients<XREG, 2>(qd.tsigns, qd.tstride, e0, qd.k, dmask, groups, lane, xr, xq,
                                      c0);
      else
        kerdock_coefficients<XREG, 1>(qd.tsigns, qd.tstride, e0, qd.k, dmask, groups, lane, xr, xq,
                                      c0);
#pragma unroll
      for (int s2 = 0; s2 < 4; ++s2) c[s2] = c0[s2];
    }
    // the gather warps must be done with this chunk's previous samples
    if (st.cc >= nchunk && !warp_wait(&sh.slot_empty[st.cs], st.ph ^ 1u, sh, cfg)) return false;
    if (lane == 0) {
#pragma unroll
      for (int s2 = 0; s2 < 8; ++s2) {
        if (s2 >= cnt) break;
        const uint32_t w = ell[s2] & dmask;
        float cv = c[s2];
        if (int64_t(ell[s2] >> qd.k) == half) cv = w < qd.n ? qd.sqrt_d * xq[w] : 0.f;
        rg.coef_s[st.cs * CR + s2] = cv;
        if (qd.coef_out) qd.coef_out[j0 + s2] = cv;
      }
      mbar_arrive(&sh.coef_full[st.cs]);
    }
    st.cs += CW;
    if (st.cs >= nchunk) {
      st.cs -= nchunk;
      st.ph ^= 1u;
    }
  }
  st.cbase = cend;
  return true;
}

// XMODE: 0 = x in registers (n <= 1024), 1 = x in shared memory, 2 = per query.
template <class Seq, int XMODE, int CW>
__device__ void coef_role(const Seq& seq, const LaunchCfg& cfg, const Regions& rg, Shared& sh) {
  const int lane = threadIdx.x & 31;
  const int cw = (threadIdx.x >> 5) - kFirstCoefWarp;
  CoefState st{uint32_t(cw), 0u, uint64_t(cw), 0};  // nchunk > CW (make_cfg)
  const int64_t nq = seq.size();
  for (int64_t qs = 0; qs < nq; ++qs) {
    const QueryDesc qd = seq.get(qs);
    const int xb = int(qs % kXBufs);
    if (!warp_wait(&sh.x_full[xb], uint32_t(qs / kXBufs) & 1u, sh, cfg)) return;
    const float* xq = rg.xbuf + xb * cfg.xpad;
    bool ok;
    if constexpr (XMODE == 0) {
      ok = coef_query<true, CW, false>(qd, qs, st, cfg, rg, sh, xq);
    } else if constexpr (XMODE == 1) {
      ok = coef_query<false, CW, false>(qd, qs, st, cfg, rg, sh, xq);
    } else {  // the batch kernel
      ok = qd.n <= 1024 ? coef_query<true, CW, true>(qd, qs, st, cfg, rg, sh, xq)
                        : coef_query<false, CW, true>(qd, qs, st, cfg, rg, sh, xq);
    }
    if (!ok) return;
    __syncwarp();
    if (lane == 0) mbar_arrive(&sh.x_empty[xb]);
  }
}

// ---------------------------------------------------------------- gather
// PACK (the batch kernel): a chunk holds crows * rows_per_slot rows.
template <typename RT, int GPT, int CW, bool PACK>
__device__ bool gather_query(const QueryDesc& qd, int64_t qs, uint32_t& cs, uint32_t& ph,
                             const LaunchCfg& cfg, const Regions& rg, Shared& sh, float* means) {
  using G = Granule<RT>;
  constexpr int GR = G::kElems;
  const int lane = threadIdx.x & 31;
  using RL = Roles<CW>;
  const int gt = threadIdx.x - RL::kFirstGatherWarp * 32;
  const int CR = cfg.crows;
  const uint32_t nchunk = uint32_t(cfg.nchunk);
  const int mb = int(qs % kMBufs);
  float2 acc[GPT][GR / 2];
#pragma unroll
  for (int u = 0; u < GPT; ++u)
#pragma unroll
    for (int e = 0; e < GR / 2; ++e) acc[u][e] = make_float2(0.f, 0.f);
  int batch_left = qd.J, batch = 0;
  const int RPC = PACK ? CR * rows_per_slot(qd, cfg) : CR;  // rows per chunk
  for (int64_t j0 = 0; j0 < qd.N; j0 += RPC) {
    const int cnt = int(qd.N - j0 < RPC ? qd.N - j0 : RPC);
    bool ok = wait_phase(&sh.row_full[cs], ph, sh, cfg);
    if (ok) ok = wait_phase(&sh.coef_full[cs], ph, sh, cfg);
    if constexpr (PACK) {
      // row s2 of the chunk at byte s2 * row_bytes of its CR slots
      const unsigned char* chunk = rg.ring + size_t(cs) * CR * cfg.slot_bytes;
      const float* cf = rg.coef_s + cs * kMaxChunkRows;
#pragma unroll 4
      for (int s2 = 0; s2 < cnt; ++s2) {
        if (!ok) break;
        const float c = cf[s2];
        const unsigned char* row = chunk + size_t(s2) * qd.row_bytes;
#pragma unroll
        for (int u = 0; u < GPT; ++u) {
          const int gi = gt + u * RL::kGatherThreads;
          if (gi * GR < qd.ldr) {
            G::fma(row + size_t(gi) * 16, make_float2(c, c), acc[u]);
          }
        }
        if (--batch_left == 0) {
          if (batch == 0 && qs >= kMBufs &&
              !wait_phase(&sh.means_empty[mb], uint32_t(qs / kMBufs - 1) & 1u, sh, cfg)) {
            ok = false;
            break;
          }
          float* mrow = means + int64_t(batch) * qd.ldr;
#pragma unroll
          for (int u = 0; u < GPT; ++u) {
            const int gi = gt + u * RL::kGatherThreads;
            if (gi * GR < qd.ldr) {
#pragma unroll
              for (int e = 0; e < GR / 2; ++e) {
                mrow[gi * GR + 2 * e] = acc[u][e].x * qd.inv_J;
                mrow[gi * GR + 2 * e + 1] = acc[u][e].y * qd.inv_J;
                acc[u][e] = make_float2(0.f, 0.f);
              }
            }
          }
          batch_left = qd.J;
          ++batch;
        }
      }
    } else {
#pragma unroll
      for (int s2 = 0; s2 < 8; ++s2) {
        if (s2 >= cnt || !ok) break;
        const float c = rg.coef_s[cs * CR + s2];
        const unsigned char* row = rg.ring + (size_t(cs) * CR + s2) * cfg.slot_bytes;
#pragma unroll
        for (int u = 0; u < GPT; ++u) {
          const int gi = gt + u * RL::kGatherThreads;
          if (gi * GR < qd.ldr) {
            G::fma(row + size_t(gi) * 16, make_float2(c, c), acc[u]);
          }
        }
        if (--batch_left == 0) {
          if (batch == 0 && qs >= kMBufs &&
              !wait_phase(&sh.means_empty[mb], uint32_t(qs / kMBufs - 1) & 1u, sh, cfg)) {
            ok = false;
            break;
          }
          float* mrow = means + int64_t(batch) * qd.ldr;
#pragma unroll
          for (int u = 0; u < GPT; ++u) {
            const int gi = gt + u * RL::kGatherThreads;
            if (gi * GR < qd.ldr) {
#pragma unroll
              for (int e = 0; e < GR / 2; ++e) {
                mrow[gi * GR + 2 * e] = acc[u][e].x * qd.inv_J;
                mrow[gi * GR + 2 * e + 1] = acc[u][e].y * qd.inv_J;
                acc[u][e] = make_float2(0.f, 0.f);
              }
            }
          }
          batch_left = qd.J;
          ++batch;
        }
      }
    }
    // the chunk's one warp-wide agreement (also where the warp reconverges
    // before the slot is freed): every lane goes on, or every lane stops
    if (!__all_sync(0xffffffffu, ok)) return false;
    __syncwarp();
    if (lane == 0) mbar_arrive(&sh.slot_empty[cs]);
    if (++cs == nchunk) {
      cs = 0;
      ph ^= 1u;
    }
  }
  return true;
}

// DYN: the representation type is chosen per query (batches of mixed plans).
template <class Seq, typename RT, int GPT, bool DYN, int CW>
__device__ void gather_role(const Seq& seq, const LaunchCfg& cfg, const Regions& rg, Shared& sh) {
  const int lane = threadIdx.x & 31;
  uint32_t cs = 0, ph = 0;
  const int64_t nq = seq.size();
  for (int64_t qs = 0; qs < nq; ++qs) {
    const QueryDesc qd = seq.get(qs);
    float* means = rg.means_base + (qs % kMBufs) * cfg.mstride;
    bool ok;
    if (DYN) {
      // each query's own type and granules per gather thread (a batch mixes
      // row sizes; the loop for the largest would idle on the smaller rows)
      constexpr int kGT = Roles<CW>::kGatherThreads;
      const int64_t gran = qd.ldr / (qd.dtype == KERDOCK_BF16 ? 8 : 4);
      const int gpt = gran <= kGT ? 1 : (gran <= 2 * kGT ? 2 : 4);
      if (qd.dtype == KERDOCK_BF16) {
        ok = gpt == 1   ? gather_query<__nv_bfloat16, 1, CW, true>(qd, qs, cs, ph, cfg, rg, sh, means)
             : gpt == 2 ? gather_query<__nv_bfloat16, 2, CW, true>(qd, qs, cs, ph, cfg, rg, sh, means)
                        : gather_query<__nv_bfloat16, GPT, CW, true>(qd, qs, cs, ph, cfg, rg, sh, means);
      } else {
        ok = gpt == 1   ? gather_query<float, 1, CW, true>(qd, qs, cs, ph, cfg, rg, sh, means)
             : gpt == 2 ? gather_query<float, 2, CW, true>(qd, qs, cs, ph, cfg, rg, sh, means)
                        : gather_query<float, GPT, CW, true>(qd, qs, cs, ph, cfg, rg, sh, means);
      }
    } else {
      ok = gather_query<RT, GPT, CW, false>(qd, qs, cs, ph, cfg, rg, sh, means);
    }
    if (!ok) return;
    if (cfg.means_gmem != nullptr) __threadfence_block();
    __syncwarp();
    if (lane == 0) mbar_arrive(&sh.means_full[qs % kMBufs]);
  }
}

// ---------------------------------------------------------------- finalizer
template <class Seq>
__device__ void final_role(const Seq& seq, const LaunchCfg& cfg, const Regions& rg, Shared& sh) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ft = tid - kFirstFinalWarp * 32;
  const int fw = warp - kFirstFinalWarp;
  float* mus = rg.mus;
  int32_t* sel = rg.sel;
  float* vals = rg.vals;
  const int64_t nq = seq.size();
  for (int64_t qs = 0; qs < nq; ++qs) {
    const QueryDesc qd = seq.get(qs);
    const int m = int(qd.m);
    const int mb = int(qs % kMBufs), xb = int(qs % kXBufs);
    {
      // the four finalizer warps stop together or go on together: each thread
      // waits, any that gave up raises the shared flag, and all read it after
      // the barrier (the flag is never lowered within a launch)
      bool ok = wait_phase(&sh.means_full[mb], uint32_t(qs / kMBufs) & 1u, sh, cfg);
      if (ok) ok = wait_phase(&sh.x_full[xb], uint32_t(qs / kXBufs) & 1u, sh, cfg);
      if (!ok) *reinterpret_cast<volatile int*>(&sh.final_abort) = 1;
      named_barrier_sync(kFinalBarrier, kFinalThreads);
      if (*reinterpret_cast<volatile int*>(&sh.final_abort)) return;
    }
    const float* means = rg.means_base + int64_t(mb) * cfg.mstride;
    const float* xq = rg.xbuf + xb * cfg.xpad;
    // a6: median over the K batch means.
    for (int col = ft; col < m; col += kFinalThreads) {
      float med;
      if (qd.K == 1) {
        med = means[col];
      } else if (qd.K == 2) {
        med = 0.5f * (means[col] + means[qd.ldr + col]);
      } else if (qd.K <= kRegK) {
        float v[kRegK];
#pragma unroll
        for (int kk = 0; kk < kRegK; ++kk) v[kk] = kk < qd.K ? means[kk * qd.ldr + col] : 0.f;
        const int r_lo = (qd.K - 1) / 2, r_hi = qd.K / 2;
        float lo = 0.f, hi = 0.f;
#pragma unroll
        for (int i = 0; i < kRegK; ++i) {
          if (i >= qd.K) break;
          int rank = 0;
#pragma unroll
          for (int j = 0; j < kRegK; ++j)
            if (j < qd.K && (v[j] < v[i] || (v[j] == v[i] && j < i))) ++rank;
          if (rank == r_lo) lo = v[i];
          if (rank == r_hi) hi = v[i];
        }
        med = (qd.K & 1) ? lo : 0.5f * (lo + hi);
      } else {
        // more batches than registers (Theorem 3's K at large m / eta): the
        // same rank selection, reading the means where they are
        const int r_lo = (qd.K - 1) / 2, r_hi = qd.K / 2;
        float lo = 0.f, hi = 0.f;
#pragma unroll 1
        for (int i = 0; i < qd.K; ++i) {
          const float vi = means[int64_t(i) * qd.ldr + col];
          int rank = 0;
#pragma unroll 4
          for (int j = 0; j < qd.K; ++j) {
            const float vj = means[int64_t(j) * qd.ldr + col];
            if (vj < vi || (vj == vi && j < i)) ++rank;
          }
          if (rank == r_lo) lo = vi;
          if (rank == r_hi) hi = vi;
        }
        med = (qd.K & 1) ? lo : 0.5f * (lo + hi);
      }
      mus[col] = med;
      if (qd.mu_out) qd.mu_out[col] = med;
    }
    named_barrier_sync(kFinalBarrier, kFinalThreads);
    if (ft == 0) mbar_arrive(&sh.means_empty[mb]);  // the means are consumed

    // a7: top-S by radix select on |mu| (4 digits of 8 bits, high first).
    uint32_t prefix = 0, mask = 0, remaining = uint32_t(qd.S);
    for (int pass = 0; pass < 4; ++pass) {
      const int shift = 24 - 8 * pass;
      for (int i = ft; i < 256; i += kFinalThreads) sh.hist[i] = 0;
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

    // a8: exact refinement v_i = a_i^T x, four rows per warp in flight.  All S
    // rows are first requested into L2 by bulk prefetches (one instruction per
    // row, no registers held), so the dot products below mostly hit L2.
    if (qd.a_vec4) {
      const uint32_t rbytes = uint32_t(qd.n) * 4u;
      for (int r = ft; r < qd.S; r += kFinalThreads)
        bulk_prefetch_l2(qd.A + int64_t(sel[r]) * qd.lda, rbytes);
    }
    for (int r0 = fw * 4; r0 < qd.S; r0 += kFinalWarps * 4) {
      float racc[4] = {0.f, 0.f, 0.f, 0.f};
      const float* arow[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        arow[u] = qd.A + int64_t(sel[r0 + u < qd.S ? r0 + u : r0]) * qd.lda;
      if (qd.a_vec4) {
        const float4* xs4 = reinterpret_cast<const float4*>(xq);
        const int n4 = int(qd.n >> 2);
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
        for (int64_t p = lane; p < qd.n; p += 32) {
          const float xv = xq[p];
#pragma unroll
          for (int u = 0; u < 4; ++u) racc[u] = fmaf(__ldg(arow[u] + p), xv, racc[u]);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float v = warp_sum(racc[u]);
        if (lane == 0 && r0 + u < qd.S) vals[r0 + u] = v;
      }
    }
    named_barrier_sync(kFinalBarrier, kFinalThreads);
    {
      const int seg = (qd.S + kFinalThreads - 1) / kFinalThreads;
      const int lo = ft * seg, hi = lo + seg < qd.S ? lo + seg : qd.S;
      const bool full = qd.flags & KERDOCK_FLAG_FULL_OUTPUT;
      int keep = 0;
      for (int r = lo; r < hi; ++r) keep += full || fabsf(vals[r]) >= qd.eps;
      int tot;
      int pos = final_exclusive_scan(keep, sh.scan, &tot);
      for (int r = lo; r < hi; ++r) {
        if (full || fabsf(vals[r]) >= qd.eps) {
          qd.out_idx[pos] = sel[r];
          qd.out_val[pos] = vals[r];
          ++pos;
        }
      }
      if (ft == 0) *qd.out_count = tot;
    }
    named_barrier_sync(kFinalBarrier, kFinalThreads);
    if (ft == 0) mbar_arrive(&sh.x_empty[xb]);  // x of this query is no longer needed
  }
}

template <class Seq, typename RT, int GPT, bool DYN, int XMODE, int CW>
__device__ __forceinline__ void run_roles(const Seq& seq, const LaunchCfg& cfg, Shared& sh,
                                          unsigned char* smem) {
  const Regions rg = regions(smem, cfg);
  init_barriers<CW>(sh, cfg);
  const int warp = threadIdx.x >> 5;
  if (warp == 0) {
    producer_role(seq, cfg, rg, sh);
  } else if (warp < Roles<CW>::kFirstGatherWarp) {
    coef_role<Seq, XMODE, CW>(seq, cfg, rg, sh);
  } else if (warp < kFirstFinalWarp) {
    gather_role<Seq, RT, GPT, DYN, CW>(seq, cfg, rg, sh);
  } else {
    final_role(seq, cfg, rg, sh);
  }
  // Every role has returned (all waits are bounded).  After an abort, row
  // copies the producer issued may still be in flight: wait, boundedly, for
  // the last arming of every ring chunk to land before the CTA's shared
  // memory is released.
  __syncthreads();
  if (threadIdx.x == 0 && *reinterpret_cast<volatile int*>(&sh.abort_flag)) {
    for (int c = 0; c < cfg.nchunk; ++c) {
      const uint32_t f = sh.armed[c];
      if (f == 0) continue;
      const uint32_t parity = ((f - 1u) / uint32_t(cfg.nchunk)) & 1u;  // phase of its last arming
      for (uint32_t it = 0; it < kDefaultPollLimit; ++it)
        if (mbar_try_wait(&sh.row_full[c], parity)) break;
    }
  }
}

// Single-plan kernel: the representation type, granules per gather thread and
// the x placement are compile-time.
template <typename RT, int GPT, bool XREG>
__global__ void __launch_bounds__(kThreads, 1) query_kernel(const QueryArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ Shared sh;
  SingleSeq seq{a};
  run_roles<SingleSeq, RT, GPT, false, XREG ? 0 : 1, coef_warps<RT, XREG>()>(seq, a.cfg, sh,
                                                                              smem);
}

// Batch kernel: any mix of plans (types and sizes), one descriptor per query.
__global__ void __launch_bounds__(kThreads, 1) query_batch_kernel(const BatchArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ Shared sh;
  BatchSeq seq{a};
  run_roles<BatchSeq, float, 4, true, 2, kCoefWarpsBatch>(seq, a.cfg, sh, smem);
}

}  // namespace

size_t align_up(size_t v, size_t al) { return (v + al - 1) / al * al; }

void dims_add(Dims& dm, const Plan& p, int64_t K, int64_t S) {
  const uint32_t rb = uint32_t(p.ldr * p.elem_bytes());
  if (rb > dm.row_bytes) dm.row_bytes = rb;
  const int64_t xp = p.d > 32 ? p.d : 32;
  if (xp > dm.xpad) dm.xpad = xp;
  if (p.ldr > dm.ldr) dm.ldr = p.ldr;
  if (S > dm.S) dm.S = S;
  if (K * p.ldr > dm.KL) dm.KL = K * p.ldr;
}

bool means_fit_smem(const Dims& dm) {
  return size_t(kMBufs) * size_t(dm.KL) * 4 <= kMeansSmemMax;
}

// Shared-memory layout for a launch.  ring_kb caps the row ring (0 = default
// 160 KiB), crows forces the rows per chunk (0 = eight when the ring holds at
// least eight such chunks, else four when it holds eight chunks of four, else
// two, else one: the chunk's barriers and waits are paid once per chunk, and
// with 2 KiB rows (n = 1024, bfloat16) chunks of eight took 0.63 ms for 1000
// queries against 0.72 ms with four).  Returns false when the ring cannot hold
// more chunks than the kernel has coefficient warps.
bool make_cfg(const Dims& dm, const Tuning& tu, bool means_in_smem, LaunchCfg& c, bool packed) {
  c = LaunchCfg{};
  c.poll_limit = kDefaultPollLimit;
  c.slot_bytes = dm.row_bytes;
  c.xpad = dm.xpad;
  c.mstride = dm.KL;
  const size_t spad = align_up(size_t(dm.S), 4);
  const size_t means_bytes = size_t(kMBufs) * size_t(dm.KL) * 4;
  const size_t fixed = size_t(kXBufs) * size_t(dm.xpad) * 4 + (means_in_smem ? means_bytes : 0) +
                       size_t(dm.ldr) * 4 + 2 * spad * 4 + 1024;
  const size_t per_slot = size_t(dm.row_bytes) + 4;
  size_t avail = kSmemBudget > fixed ? kSmemBudget - fixed : 0;
  const size_t ring_cap = (tu.ring_kb > 0 ? size_t(tu.ring_kb) << 10 : kRingCap);
  const size_t cap = ring_cap + size_t(kMaxSlots) * 4;
  if (avail > cap) avail = cap;
  int ns = int(avail / per_slot);
  if (ns > kMaxSlots) ns = kMaxSlots;
  const int min_chunks = dm.coef_warps + 1;
  int cr = tu.crows > 0 ? tu.crows
                        : (ns >= 64 ? 8 : ns >= 32 ? 4 : ns >= 2 * min_chunks ? 2 : 1);
  if (cr != 1 && cr != 2 && cr != 4 && cr != 8) return false;
  c.crows = cr;
  c.nchunk = ns / cr;
  if (c.nchunk < min_chunks) return false;
  if (c.nchunk > kMaxChunks) c.nchunk = kMaxChunks;
  // the layout; with packed chunks the coefficients take kMaxChunkRows floats
  // per chunk, and a ring that leaves no room for them loses chunks
  for (;; --c.nchunk) {
    if (c.nchunk < min_chunks) return false;
    ns = c.nchunk * cr;
    size_t off = align_up(size_t(ns) * dm.row_bytes, 128);
    c.off_coef = uint32_t(off);
    off = align_up(off + (packed ? size_t(c.nchunk) * kMaxChunkRows : size_t(ns)) * 4, 16);
    c.off_x = uint32_t(off);
    off = align_up(off + size_t(kXBufs) * size_t(dm.xpad) * 4, 16);
    c.off_means = uint32_t(off);
    if (means_in_smem) off = align_up(off + means_bytes, 16);
    c.off_mu = uint32_t(off);
    off = align_up(off + size_t(dm.ldr) * 4, 16);
    c.off_sel = uint32_t(off);
    off = align_up(off + spad * 4, 16);
    c.off_vals = uint32_t(off);
    off = align_up(off + spad * 4, 16);
    c.total = uint32_t(off);
    if (off <= kSmemBudget) break;
    if (!packed) return false;
  }
  int g = 1;  // chunks per producer step: g * crows <= 32 lanes, g <= nchunk / 2
  while (2 * g * cr <= 32 && 4 * g <= c.nchunk) g *= 2;
  c.pgroup = g;
  return true;
}

// Descriptor fields that come from the plan alone.
QueryDesc plan_desc(const Plan& p) {
  QueryDesc d{};
  d.R = p.repr;
  d.tsigns = p.tsigns();
  d.A = p.A;
  d.tstride = p.tsign_words;
  d.lda = p.lda;
  d.m = p.m;
  d.n = p.n;
  d.d = p.d;
  d.L = p.L;
  d.ldr = p.ldr;
  d.k = p.k;
  d.dtype = p.dtype;
  d.a_vec4 =
      (p.n % 4 == 0 && p.lda % 4 == 0 && (reinterpret_cast<uintptr_t>(p.A) & 15) == 0) ? 1 : 0;
  d.row_bytes = uint32_t(p.ldr * p.elem_bytes());
  d.sqrt_d = float(int64_t(1) << (p.k / 2));
  return d;
}

void set_query_params(QueryDesc& d, int64_t J, int64_t K, int64_t S, float eps, uint64_t seed,
                      int flags) {
  d.J = int32_t(J);
  d.K = int32_t(K);
  d.N = J * K;
  d.S = int32_t(S);
  d.eps = eps;
  d.inv_J = 1.0f / float(J);
  d.seed = seed;
  d.flags = flags;
}

namespace {

template <typename RT, int GPT, bool XREG>
int launch_single(const QueryArgs& a, int64_t grid, cudaStream_t stream) {
  auto kern = query_kernel<RT, GPT, XREG>;
  // The cap is one per kernel for the whole process, graphs captured by a
  // caller included: set to the largest layout (make_cfg's budget), never to
  // this launch's size, which would make a captured launch of a plan with a
  // larger layout fail.
  KD_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   int(kSmemBudget)));
  kern<<<unsigned(grid), kThreads, a.cfg.total, stream>>>(a);
  KD_CUDA_TRY(cudaGetLastError());
  return KERDOCK_OK;
}

// Granules (16 bytes) per gather thread: the row's granules over the gather
// threads of the role split used for this n (m <= 4096 and 256 gather threads
// bound it by 4).
int dispatch_single(const Plan& p, const QueryArgs& a, int64_t grid) {
  const int64_t granule = 16 / int64_t(p.elem_bytes());
  const bool xreg = p.n <= 1024;
  const bool bf = p.dtype == KERDOCK_BF16;
  const int64_t gthreads =
      xreg ? (bf ? Roles<coef_warps<__nv_bfloat16, true>()>::kGatherThreads
                 : Roles<coef_warps<float, true>()>::kGatherThreads)
           : (bf ? Roles<coef_warps<__nv_bfloat16, false>()>::kGatherThreads
                 : Roles<coef_warps<float, false>()>::kGatherThreads);
  const int64_t gpt = (p.ldr / granule + gthreads - 1) / gthreads;
  if (p.dtype == KERDOCK_BF16) {
    if (gpt <= 1) return xreg ? launch_single<__nv_bfloat16, 1, true>(a, grid, p.stream)
                              : launch_single<__nv_bfloat16, 1, false>(a, grid, p.stream);
    if (gpt <= 2) return xreg ? launch_single<__nv_bfloat16, 2, true>(a, grid, p.stream)
                              : launch_single<__nv_bfloat16, 2, false>(a, grid, p.stream);
    if (gpt <= 4 && !xreg) return launch_single<__nv_bfloat16, 4, false>(a, grid, p.stream);
    return KERDOCK_ERR_UNSUPPORTED;
  }
  if (gpt <= 1) return xreg ? launch_single<float, 1, true>(a, grid, p.stream)
                            : launch_single<float, 1, false>(a, grid, p.stream);
  if (gpt <= 2) return xreg ? launch_single<float, 2, true>(a, grid, p.stream)
                            : launch_single<float, 2, false>(a, grid, p.stream);
  if (gpt <= 4) return xreg ? launch_single<float, 4, true>(a, grid, p.stream)
                            : launch_single<float, 4, false>(a, grid, p.stream);
  return KERDOCK_ERR_UNSUPPORTED;
}

}  // namespace

Dims plan_dims(const Plan& p) {
  Dims dm;
  dims_add(dm, p, p.K, p.S);
  const bool bf = p.dtype == KERDOCK_BF16;
  dm.coef_warps = p.n > 1024 ? (bf ? coef_warps<__nv_bfloat16, false>() : coef_warps<float, false>())
                             : (bf ? coef_warps<__nv_bfloat16, true>() : coef_warps<float, true>());
  return dm;
}

size_t apply_workspace_bytes(const Plan& p, int64_t q) {
  const Dims dm = plan_dims(p);
  if (means_fit_smem(dm) || q == 0) return 0;
  const int64_t grid = p.num_sms > 0 ? p.num_sms : 256;
  return size_t(grid) * kMBufs * size_t(dm.KL) * 4;
}

int launch_apply(const Plan& p, const float* X, int64_t q, int64_t ldx, float eps, uint64_t seed,
                 int flags, int32_t* out_idx, float* out_val, int32_t* out_count, void* ws,
                 size_t ws_bytes, float* mu_out, int64_t* ells_out, float* coef_out) {
  (void)ws_bytes;
  const Dims dm = plan_dims(p);
  const bool smem_means = means_fit_smem(dm);
  QueryArgs a{};
  if (!make_cfg(dm, p.tuning, smem_means, a.cfg)) return KERDOCK_ERR_UNSUPPORTED;
  a.cfg.means_gmem = smem_means ? nullptr : static_cast<float*>(ws);
  a.cfg.status = p.status();
  a.cfg.poll_limit = p.poll_limit;
  a.base = plan_desc(p);
  set_query_params(a.base, p.J, p.K, p.S, eps, seed, flags);
  a.base.x = X;
  a.base.out_idx = out_idx;
  a.base.out_val = out_val;
  a.base.out_count = out_count;
  a.base.mu_out = mu_out;
  a.base.ells_out = ells_out;
  a.base.coef_out = coef_out;
  a.Q = q;
  a.ldx = ldx;
  int64_t grid = p.num_sms;
  if (grid > q) grid = q;
  return dispatch_single(p, a, grid);
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

}  // namespace

size_t noalloc_scratch_bytes() { return kNoAllocScratchBytes; }

int launch_apply_noalloc(const Plan& p, const float* X, int64_t q, int64_t ldx, float eps,
                         uint64_t seed, int flags, int32_t* out_idx, float* out_val,
                         int32_t* out_count) {
  const Dims dm = plan_dims(p);
  QueryArgs a{};
  // the batch means always go to the scratch array, so the whole shared-memory
  // budget goes to the row ring
  if (!make_cfg(dm, p.tuning, false, a.cfg)) return KERDOCK_ERR_UNSUPPORTED;
  int64_t grid = p.num_sms;
  if (grid > q) grid = q;
  const size_t need = size_t(grid) * kMBufs * size_t(dm.KL) * sizeof(float);
  if (need > kNoAllocScratchBytes) return KERDOCK_ERR_CAPACITY;  // beyond the fixed scratch
  void* scratch = nullptr;
  const int rc = noalloc_scratch(&scratch);
  if (rc != KERDOCK_OK) return rc;
  a.cfg.means_gmem = static_cast<float*>(scratch);
  a.cfg.status = p.status();
  a.cfg.poll_limit = p.poll_limit;
  a.base = plan_desc(p);
  set_query_params(a.base, p.J, p.K, p.S, eps, seed, flags);
  a.base.x = X;
  a.base.out_idx = out_idx;
  a.base.out_val = out_val;
  a.base.out_count = out_count;
  a.Q = q;
  a.ldx = ldx;
  return dispatch_single(p, a, grid);
}

// ---------------------------------------------------------------------------
// Batches of queries over any mix of plans (one persistent launch).
// ---------------------------------------------------------------------------
int prepare_batch_kernel(const LaunchCfg& cfg) {
  // One cap for every batch (each batch's graph keeps its own layout size):
  // the largest layout, so that a batch configured later with a smaller one
  // does not make the others' launches fail.
  if (cfg.total > kSmemBudget) return KERDOCK_ERR_UNSUPPORTED;
  KD_CUDA_TRY(cudaFuncSetAttribute(query_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   int(kSmemBudget)));
  return KERDOCK_OK;
}

int launch_batch(const LaunchCfg& cfg, const QueryDesc* descs, const int32_t* order,
                 const int64_t* cta_start, int grid, cudaStream_t stream) {
  BatchArgs a{};
  a.cfg = cfg;
  a.descs = descs;
  a.order = order;
  a.cta_start = cta_start;
  query_batch_kernel<<<unsigned(grid), kThreads, cfg.total, stream>>>(a);
  KD_CUDA_TRY(cudaGetLastError());
  return KERDOCK_OK;
}

}  // namespace kd
