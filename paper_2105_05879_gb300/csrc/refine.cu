// refine.cu -- Algorithm 1's last two steps driven by arbitrary candidate
// scores: take the S indices with the largest scores (ties to the smaller
// index), compute A_S x exactly and keep |value| >= eps.  Used by the learned
// proposal, whose network scores replace |mu|.
#include "kerdock_internal.cuh"

namespace kd {
namespace {

constexpr int kRThreads = 128;
constexpr int kRWarps = kRThreads / 32;

// Order-preserving map from float to uint32 (larger float -> larger key).
__device__ __forceinline__ uint32_t ordered_key(float v) {
  const uint32_t b = __float_as_uint(v);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ int cta_exclusive_scan(int v, int* scratch, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) scratch[warp] = x;
  __syncthreads();
  int before = 0, tot = 0;
#pragma unroll
  for (int w = 0; w < kRWarps; ++w) {
    const int s = scratch[w];
    if (w < warp) before += s;
    tot += s;
  }
  *total = tot;
  __syncthreads();
  return before + x - v;
}

struct RefineArgs {
  const float* A;
  int64_t lda, m, n;
  const float* X;
  int64_t ldx, Q;
  const float* scores;  // Q x m
  int S, flags, a_vec4;
  int64_t xs_off;  // byte offset of the staged query in shared memory (16-aligned)
  float eps;
  int32_t* out_idx;
  float* out_val;
  int32_t* out_count;
};

__global__ void __launch_bounds__(kRThreads, 4) score_refine_kernel(const RefineArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* keys = reinterpret_cast<uint32_t*>(smem);
  int32_t* sel = reinterpret_cast<int32_t*>(keys + a.m);
  float* vals = reinterpret_cast<float*>(sel + a.S);
  float* xs = reinterpret_cast<float*>(smem + a.xs_off);
  __shared__ uint32_t hist[256];
  __shared__ int scan[kRWarps];
  __shared__ uint32_t s_digit, s_remaining;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m = int(a.m);
  for (int64_t q = blockIdx.x; q < a.Q; q += gridDim.x) {
    const float* sc = a.scores + q * a.m;
    for (int i = tid; i < m; i += kRThreads) keys[i] = ordered_key(sc[i]);
    // the query is read from global memory once and kept next to the keys:
    // every row group of the refinement below reads it again
    const float* xg = a.X + q * a.ldx;
    for (int64_t p = tid; p < a.n; p += kRThreads) xs[p] = xg[p];
    __syncthreads();
    uint32_t prefix = 0, mask = 0, remaining = uint32_t(a.S);
    for (int pass = 0; pass < 4; ++pass) {
      const int shift = 24 - 8 * pass;
      hist[tid] = 0;
      hist[tid + kRThreads] = 0;
      __syncthreads();
      for (int i = tid; i < m; i += kRThreads)
        if ((keys[i] & mask) == prefix) atomicAdd(&hist[(keys[i] >> shift) & 255u], 1u);
      __syncthreads();
      if (warp == 0) {
        const int base = (31 - lane) * 8;  // lane 0 holds the highest digits
        uint32_t sum = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) sum += hist[base + j];
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
          for (int j = 7; j >= 0; --j) {
            const uint32_t h = hist[base + j];
            if (cum + h >= remaining) {
              s_digit = uint32_t(base + j);
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
    const uint32_t T = prefix;
    {
      const int seg = (m + kRThreads - 1) / kRThreads;
      const int lo = tid * seg, hi = lo + seg < m ? lo + seg : m;
      int eq = 0;
      for (int i = lo; i < hi; ++i) eq += keys[i] == T;
      int tot;
      int eq_rank = cta_exclusive_scan(eq, scan, &tot);
      const int eq_rank0 = eq_rank;
      int take = 0;
      for (int i = lo; i < hi; ++i) {
        if (keys[i] > T) {
          ++take;
        } else if (keys[i] == T) {
          take += uint32_t(eq_rank) < remaining;
          ++eq_rank;
        }
      }
      int pos = cta_exclusive_scan(take, scan, &tot);
      eq_rank = eq_rank0;
      for (int i = lo; i < hi; ++i) {
        bool t2 = false;
        if (keys[i] > T) {
          t2 = true;
        } else if (keys[i] == T) {
          t2 = uint32_t(eq_rank) < remaining;
          ++eq_rank;
        }
        if (t2) sel[pos++] = i;
      }
    }
    __syncthreads();
    if (a.a_vec4) {  // all S rows requested into L2 up front (no registers held)
      const uint32_t rbytes = uint32_t(a.n) * 4u;
      for (int r = tid; r < a.S; r += kRThreads) bulk_prefetch_l2(a.A + int64_t(sel[r]) * a.lda, rbytes);
    }
    const float* x = xs;
    const bool xv4 = a.a_vec4;
    for (int r0 = warp * 4; r0 < a.S; r0 += kRWarps * 4) {
      float racc[4] = {0.f, 0.f, 0.f, 0.f};
      const float* arow[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) arow[u] = a.A + int64_t(sel[r0 + u < a.S ? r0 + u : r0]) * a.lda;
      if (xv4) {
        // four 16-byte pieces of each of the four rows requested before any
        // is used (20 loads in flight per lane against the L2 latency), then
        // the tail piece by piece; the sum order is p4 = lane, lane + 32, ...
        const int n4 = int(a.n >> 2);
        const float4* xp = reinterpret_cast<const float4*>(x);
        int p4 = lane;
        for (; p4 + 96 < n4; p4 += 128) {
          float4 xq[4], av[4][4];
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            xq[t] = xp[p4 + 32 * t];
#pragma unroll
            for (int u = 0; u < 4; ++u)
              av[u][t] = __ldg(reinterpret_cast<const float4*>(arow[u]) + p4 + 32 * t);
          }
#pragma unroll
          for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              racc[u] = fmaf(av[u][t].x, xq[t].x, racc[u]);
              racc[u] = fmaf(av[u][t].y, xq[t].y, racc[u]);
              racc[u] = fmaf(av[u][t].z, xq[t].z, racc[u]);
              racc[u] = fmaf(av[u][t].w, xq[t].w, racc[u]);
            }
        }
        for (; p4 < n4; p4 += 32) {
          const float4 xq = xp[p4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float4 av = __ldg(reinterpret_cast<const float4*>(arow[u]) + p4);
            racc[u] = fmaf(av.x, xq.x, racc[u]);
            racc[u] = fmaf(av.y, xq.y, racc[u]);
            racc[u] = fmaf(av.z, xq.z, racc[u]);
            racc[u] = fmaf(av.w, xq.w, racc[u]);
          }
        }
      } else {
        for (int64_t p = lane; p < a.n; p += 32) {
          const float xv = x[p];
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
      const int seg = (a.S + kRThreads - 1) / kRThreads;
      const int lo = tid * seg, hi = lo + seg < a.S ? lo + seg : a.S;
      const bool full = a.flags & KERDOCK_FLAG_FULL_OUTPUT;
      int keep = 0;
      for (int r = lo; r < hi; ++r) keep += full || fabsf(vals[r]) >= a.eps;
      int tot;
      int pos = cta_exclusive_scan(keep, scan, &tot);
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
    __syncthreads();
  }
}

}  // namespace
}  // namespace kd

extern "C" int kerdock_refine_scores(kerdock_plan_t plan, const float* X_dev, int64_t q,
                                     int64_t ldx, const float* scores, int32_t S, float eps,
                                     int32_t flags, int32_t* out_idx, float* out_val,
                                     int32_t* out_count) {
  if (plan == nullptr || q < 0) return KERDOCK_ERR_INVALID_ARG;
  const kd::Plan& p = plan->p;
  if (!p.bound) return KERDOCK_ERR_NOT_BOUND;
  if (!p.preprocessed) return KERDOCK_ERR_NOT_PREPROCESSED;
  if (q == 0) return KERDOCK_OK;
  if (X_dev == nullptr || scores == nullptr || out_idx == nullptr || out_val == nullptr ||
      out_count == nullptr || ldx < p.n)
    return KERDOCK_ERR_INVALID_ARG;
  if (S < 1 || S > p.m || flags < 0 || flags > KERDOCK_FLAG_FULL_OUTPUT)
    return KERDOCK_ERR_INVALID_ARG;
  if (!(flags & KERDOCK_FLAG_FULL_OUTPUT) && !(eps > 0.0f)) return KERDOCK_ERR_INVALID_ARG;
  kd::RefineArgs a{};
  a.A = p.A;
  a.lda = p.lda;
  a.m = p.m;
  a.n = p.n;
  a.X = X_dev;
  a.ldx = ldx;
  a.Q = q;
  a.scores = scores;
  a.S = S;
  a.flags = flags;
  a.a_vec4 =
      (p.n % 4 == 0 && p.lda % 4 == 0 && (reinterpret_cast<uintptr_t>(p.A) & 15) == 0) ? 1 : 0;
  a.eps = eps;
  a.out_idx = out_idx;
  a.out_val = out_val;
  a.out_count = out_count;
  a.xs_off = int64_t((size_t(p.m) * 4 + size_t(S) * 8 + 15) / 16 * 16);
  const size_t smem = size_t(a.xs_off) + size_t(p.n) * 4;
  // the cap is per kernel and process-wide (captured graphs included): the
  // largest layout, m = S = n = 4096, never this launch's size
  constexpr int kCap = (4096 * 4 + 4096 * 8) + 4096 * 4;
  if (smem > size_t(kCap)) return KERDOCK_ERR_UNSUPPORTED;
  KD_CUDA_TRY(cudaFuncSetAttribute(kd::score_refine_kernel,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, kCap));
  int64_t grid = int64_t(p.num_sms) * 8;
  if (grid > q) grid = q;
  kd::score_refine_kernel<<<unsigned(grid), kd::kRThreads, smem, p.stream>>>(a);
  KD_CUDA_TRY(cudaGetLastError());
  return KERDOCK_OK;
}
