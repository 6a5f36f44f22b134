// shared.cu -- Algorithm 1's streaming step with one sample set shared by a
// batch of queries.
//
// Every query of the batch uses the same N = JK indices l_j (those that
// kerdock_apply draws for query 0).  Each query is still Algorithm 1 with N
// independent uniform samples, so Theorem 3 holds per query; only the queries'
// failure events become dependent.  Sharing turns the two sums of the
// streaming step into dense products over the batch:
//   C  = X S^T          (q x N: c_qj = s_{l_j}^T x_q, Algorithm 1)
//   Y_k = C_k R_k / J   (q x m per batch k: the batch means of Theorem 3)
// where S holds the N sample vectors (+-1, or sqrt(d) e_w for the identity
// basis) and R_k the N/K gathered representation rows of batch k.  Both run on
// the tensor cores with bfloat16 operands and float32 accumulation; float32
// factors are split as hi + lo (hi = bf16(v), lo = bf16(v - hi)) so that the
// products keep about 16 significant bits (C S^T: x_hi, x_lo against exact
// +-1; C R: C_hi R_hi + C_lo R_hi + C_hi R_lo, or C_hi R + C_lo R for a
// bfloat16 representation).  The entrywise median over the K batch means, the
// top-S of |mu| and the exact refinement with the threshold (a6-a8) follow.
#include "kerdock_internal.cuh"

extern "C" int kerdock_refine_scores(kerdock_plan_t plan, const float* X_dev, int64_t q,
                                     int64_t ldx, const float* scores, int32_t S, float eps,
                                     int32_t flags, int32_t* out_idx, float* out_val,
                                     int32_t* out_count);

namespace kd {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(v);
  lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

// l_j and the sample vector s_{l_j} (restricted to the first n coordinates,
// Algorithm 1's Pi), twice per row: S2[j] = [s | s] against X2 = [x_hi | x_lo].
__global__ void shared_samples_kernel(uint64_t seed, int64_t N, int64_t L, int kbits, int64_t n,
                                      const uint32_t* __restrict__ signs, int64_t sign_words,
                                      float sqrt_d, int64_t* ells, __nv_bfloat16* S2) {
  const int64_t d = int64_t(1) << kbits;
  for (int64_t j = blockIdx.x; j < N; j += gridDim.x) {
    const uint64_t l = sample_index(seed, uint64_t(j), uint64_t(L));
    if (threadIdx.x == 0) ells[j] = int64_t(l);
    const int64_t b = int64_t(l >> kbits), w = int64_t(l & uint64_t(d - 1));
    __nv_bfloat16* row = S2 + j * 2 * n;
    for (int64_t p = threadIdx.x; p < n; p += blockDim.x) {
      float v;
      if (b == d / 2) {
        v = p == w ? sqrt_d : 0.f;
      } else {
        const uint32_t bit = (__ldg(signs + b * sign_words + (p >> 5)) >> (p & 31)) & 1u;
        const uint32_t par = uint32_t(__popcll(uint64_t(w) & uint64_t(p))) & 1u;
        v = (bit ^ par) ? -1.f : 1.f;
      }
      row[p] = __float2bfloat16_rn(v);
      row[n + p] = __float2bfloat16_rn(v);
    }
  }
}

// X2[r] = [x_hi | x_lo] for every query row.
__global__ void split_queries_kernel(const float* __restrict__ X, int64_t q, int64_t ldx,
                                     int64_t n, __nv_bfloat16* X2) {
  for (int64_t r = blockIdx.x; r < q; r += gridDim.x)
    for (int64_t p = threadIdx.x; p < n; p += blockDim.x) {
      __nv_bfloat16 hi, lo;
      split_bf16(X[r * ldx + p], hi, lo);
      X2[r * 2 * n + p] = hi;
      X2[r * 2 * n + n + p] = lo;
    }
}

// Per batch k the P copies of its J gathered rows stacked along the
// contraction index, stored k-major for the product (G3[k][i][t], t the
// contraction index, row pitch lda3): float32 rows as [R_hi | R_hi | R_lo],
// bfloat16 rows as [R | R].  A CTA moves 32 samples x 64 entries through
// shared memory, reading each row run and writing each t run contiguously.
__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename RT>
__global__ void gather_rows_kernel(const RT* __restrict__ R, int64_t ldr, const int64_t* ells,
                                   int64_t J, int64_t m, int64_t lda3, __nv_bfloat16* G3) {
  constexpr int P = sizeof(RT) == 4 ? 3 : 2;
  __shared__ float tile[32][65];
  __shared__ int64_t row_off[32];
  const int64_t k = blockIdx.z, j0 = int64_t(blockIdx.y) * 32, i0 = int64_t(blockIdx.x) * 64;
  if (threadIdx.x < 32)
    row_off[threadIdx.x] = j0 + threadIdx.x < J ? ells[k * J + j0 + threadIdx.x] * ldr : -1;
  __syncthreads();
#pragma unroll 4
  for (int e = threadIdx.x; e < 32 * 64; e += blockDim.x) {
    const int jj = e >> 6, ii = e & 63;
    const int64_t i = i0 + ii;
    tile[jj][ii] = (row_off[jj] >= 0 && i < m) ? to_f32(R[row_off[jj] + i]) : 0.f;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 32 * 64; e += blockDim.x) {
    const int jj = e & 31, ii = e >> 5;
    const int64_t j = j0 + jj, i = i0 + ii;
    if (j >= J || i >= m) continue;
    __nv_bfloat16* dst = G3 + (k * ldr + i) * lda3;
    if (P == 3) {
      __nv_bfloat16 hi, lo;
      split_bf16(tile[jj][ii], hi, lo);
      dst[j] = hi;
      dst[J + j] = hi;
      dst[2 * J + j] = lo;
    } else {
      const __nv_bfloat16 v = __float2bfloat16_rn(tile[jj][ii]);  // exact: R is bfloat16
      dst[j] = v;
      dst[J + j] = v;
    }
  }
}

// A3[k][r] = P pieces of C[r][batch k] / J: float32 [c_hi | c_lo | c_hi],
// bfloat16 [c_hi | c_lo].
// C arrives as `slices` partial planes of q x N (a split product), summed here
// in plane order.
__global__ void split_coef_kernel(const float* __restrict__ C, int slices, int64_t q, int64_t N,
                                  int64_t J, int64_t K, int P, int64_t lda3, float inv_J,
                                  __nv_bfloat16* A3) {
  for (int64_t r = blockIdx.x; r < q; r += gridDim.x)
    for (int64_t j = threadIdx.x; j < N; j += blockDim.x) {
      const int64_t k = j / J, jj = j - k * J;
      float c = 0.f;
      for (int z = 0; z < slices; ++z) c += C[(z * q + r) * N + j];
      __nv_bfloat16 hi, lo;
      split_bf16(c * inv_J, hi, lo);
      __nv_bfloat16* a = A3 + (k * q + r) * lda3;
      a[jj] = hi;
      a[J + jj] = lo;
      if (P == 3) a[2 * J + jj] = hi;
    }
}

// Median of v[0 .. K) (mean of the two middle values for even K).
template <int KM>
__device__ __forceinline__ float median_of(const float (&v)[KM], int K) {
  if (K == 1) return v[0];
  if (K == 2) return 0.5f * (v[0] + v[1]);
  const int r_lo = (K - 1) / 2, r_hi = K / 2;
  float lo = 0.f, hi = 0.f;
#pragma unroll
  for (int a = 0; a < KM; ++a) {
    if (a >= K) break;
    int rank = 0;
#pragma unroll
    for (int c = 0; c < KM; ++c)
      if (c < K && (v[c] < v[a] || (v[c] == v[a] && c < a))) ++rank;
    if (rank == r_lo) lo = v[a];
    if (rank == r_hi) hi = v[a];
  }
  return (K & 1) ? lo : 0.5f * (lo + hi);
}

// scores = |median over the K batch means| (mean of the two middle values for
// even K), q x m, four consecutive entries per thread (16-byte loads: the row
// pitch ldr is a multiple of 8).  Batch k's mean arrives as `slices` partial
// planes Y[k * slices + z] of q x ldr, summed in plane order.  KM >= K sizes
// the per-thread arrays.
template <int KM>
__global__ void median_abs_kernel(const float* __restrict__ Y, int slices, int64_t q, int64_t m,
                                  int64_t ldr, int K, float* scores) {
  const int64_t m4 = (m + 3) / 4, total = q * m4;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = t / m4, i = (t - r * m4) * 4;
    float4 y[KM];
#pragma unroll
    for (int k = 0; k < KM; ++k)
      y[k] = k < K ? *reinterpret_cast<const float4*>(Y + (int64_t(k) * slices * q + r) * ldr + i)
                   : make_float4(0.f, 0.f, 0.f, 0.f);
    for (int z = 1; z < slices; ++z)  // the other planes, added in plane order
#pragma unroll
      for (int k = 0; k < KM; ++k)
        if (k < K) {
          const float4 w =
              *reinterpret_cast<const float4*>(Y + ((int64_t(k) * slices + z) * q + r) * ldr + i);
          y[k].x += w.x;
          y[k].y += w.y;
          y[k].z += w.z;
          y[k].w += w.w;
        }
    float v[KM];
    float4 out;
#pragma unroll
    for (int k = 0; k < KM; ++k) v[k] = y[k].x;
    out.x = fabsf(median_of(v, K));
#pragma unroll
    for (int k = 0; k < KM; ++k) v[k] = y[k].y;
    out.y = fabsf(median_of(v, K));
#pragma unroll
    for (int k = 0; k < KM; ++k) v[k] = y[k].z;
    out.z = fabsf(median_of(v, K));
#pragma unroll
    for (int k = 0; k < KM; ++k) v[k] = y[k].w;
    out.w = fabsf(median_of(v, K));
    if ((m & 3) == 0) {
      *reinterpret_cast<float4*>(scores + r * m + i) = out;
    } else {
      const float o[4] = {out.x, out.y, out.z, out.w};
      for (int c = 0; c < 4 && i + c < m; ++c) scores[r * m + i + c] = o[c];
    }
  }
}

// Row stride of A3: P * J rounded up to 8 elements so that every row starts on
// a 16-byte boundary (the padding is never read: the GEMM's K is P * J).
int64_t a3_stride(int64_t P, int64_t J) { return (P * J + 7) / 8 * 8; }

struct SharedLayout {
  size_t ells, S2, X2, C, A3, G3, Y, scores, total;
  GemmSplit split_c, split_y;  // K splits of C = X S^T and of each Y_k = C_k R_k / J
};

SharedLayout shared_layout(const Plan& p, int64_t q) {
  const int64_t N = p.N, J = p.J, K = p.K, n = p.n, m = p.m, ldr = p.ldr;
  const int64_t P = p.dtype == KERDOCK_BF16 ? 2 : 3;
  SharedLayout s{};
  s.split_c = gemm_split(q, N, 2 * n, p.num_sms);
  // The batch-mean products stay whole: split three ways at q = 1000,
  // m = 1024 they ran no faster (14.3 vs 14.0 us) and their partial planes
  // tripled what the median reads.
  s.split_y = GemmSplit{1, 0};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = align_up(off + bytes, 256);
    return at;
  };
  s.ells = take(size_t(N) * 8);
  s.S2 = take(size_t(N) * 2 * n * 2);
  s.X2 = take(size_t(q) * 2 * n * 2);
  s.C = take(size_t(s.split_c.slices) * q * N * 4);
  s.A3 = take(size_t(K) * q * a3_stride(P, J) * 2);
  s.G3 = take(size_t(K) * ldr * a3_stride(P, J) * 2);
  s.Y = take(size_t(K) * s.split_y.slices * q * ldr * 4);
  s.scores = take(size_t(q) * m * 4);
  s.total = off;
  return s;
}

unsigned grid_for(int64_t units) {
  return unsigned(units < 1 ? 1 : (units > 65535 ? 65535 : units));
}

}  // namespace
}  // namespace kd

extern "C" size_t kerdock_apply_shared_workspace_bytes(kerdock_plan_t plan, int64_t q) {
  if (plan == nullptr || q <= 0) return 0;
  return kd::shared_layout(plan->p, q).total;
}

namespace kd {
namespace {

// Steps a3-a6 with the shared sample set: scores[r * m + i] = |mu_r[i]|, the
// entrywise median over the K batch means of query r (q x m, row pitch m).
// The intermediate products live in the workspace at base (layout lay).
int shared_scores(Plan& p, const float* X_dev, int64_t q, int64_t ldx, uint64_t seed, char* base,
                  const SharedLayout& lay, float* scores) {
  int64_t* ells = reinterpret_cast<int64_t*>(base + lay.ells);
  __nv_bfloat16* S2 = reinterpret_cast<__nv_bfloat16*>(base + lay.S2);
  __nv_bfloat16* X2 = reinterpret_cast<__nv_bfloat16*>(base + lay.X2);
  float* C = reinterpret_cast<float*>(base + lay.C);
  __nv_bfloat16* A3 = reinterpret_cast<__nv_bfloat16*>(base + lay.A3);
  __nv_bfloat16* G3 = reinterpret_cast<__nv_bfloat16*>(base + lay.G3);
  float* Y = reinterpret_cast<float*>(base + lay.Y);
  const int64_t N = p.N, J = p.J, K = p.K, n = p.n, m = p.m, ldr = p.ldr;
  const int P = p.dtype == KERDOCK_BF16 ? 2 : 3;
  cudaStream_t st = p.stream;

  shared_samples_kernel<<<grid_for(N), kThreads, 0, st>>>(
      seed, N, p.L, p.k, n, p.signs(), p.sign_words, float(int64_t(1) << (p.k / 2)), ells, S2);
  KD_CUDA_TRY(cudaGetLastError());
  split_queries_kernel<<<grid_for(q), kThreads, 0, st>>>(X_dev, q, ldx, n, X2);
  KD_CUDA_TRY(cudaGetLastError());
  const int64_t lda3 = a3_stride(P, J);
  const dim3 ggrid(unsigned((m + 63) / 64), unsigned((J + 31) / 32), unsigned(K));
  if (P == 3)
    gather_rows_kernel<float><<<ggrid, kThreads, 0, st>>>(static_cast<const float*>(p.repr), ldr,
                                                          ells, J, m, lda3, G3);
  else
    gather_rows_kernel<__nv_bfloat16><<<ggrid, kThreads, 0, st>>>(
        static_cast<const __nv_bfloat16*>(p.repr), ldr, ells, J, m, lda3, G3);
  KD_CUDA_TRY(cudaGetLastError());
  // C = X S^T over [x_hi | x_lo] and [s | s]
  GemmArgs g1{int(q), int(N), int(2 * n), X2, 2 * n, 1, S2, 2 * n, 1};
  g1.status = p.status();
  int rc = gemm_bf16_f32_split(g1, lay.split_c, C, N, q * N, st);
  if (rc != KERDOCK_OK) return rc;
  split_coef_kernel<<<grid_for(q), kThreads, 0, st>>>(C, lay.split_c.slices, q, N, J, K, P, lda3,
                                                      1.0f / float(J), A3);
  KD_CUDA_TRY(cudaGetLastError());
  for (int64_t k = 0; k < K; ++k) {  // Y_k = C_k R_k / J
    GemmArgs g2{int(q), int(m), int(P * J), A3 + k * q * lda3, lda3, 1, G3 + k * ldr * lda3, lda3,
                1};
    g2.status = p.status();
    rc = gemm_bf16_f32_split(g2, lay.split_y, Y + k * lay.split_y.slices * q * ldr, ldr, q * ldr,
                             st);
    if (rc != KERDOCK_OK) return rc;
  }
  const unsigned mgrid = grid_for((q * ((m + 3) / 4) + kThreads - 1) / kThreads);
  const int sl = lay.split_y.slices;
  if (K <= 2)
    median_abs_kernel<2><<<mgrid, kThreads, 0, st>>>(Y, sl, q, m, ldr, int(K), scores);
  else if (K <= 4)
    median_abs_kernel<4><<<mgrid, kThreads, 0, st>>>(Y, sl, q, m, ldr, int(K), scores);
  else if (K <= 8)
    median_abs_kernel<8><<<mgrid, kThreads, 0, st>>>(Y, sl, q, m, ldr, int(K), scores);
  else
    median_abs_kernel<kMaxK><<<mgrid, kThreads, 0, st>>>(Y, sl, q, m, ldr, int(K), scores);
  KD_CUDA_TRY(cudaGetLastError());
  return KERDOCK_OK;
}

// The checks both entry points share; on success *lay is the workspace layout.
int shared_validate(Plan& p, const float* X_dev, int64_t q, int64_t ldx, void* ws,
                    size_t ws_bytes, SharedLayout* lay) {
  if (X_dev == nullptr || ldx < p.n) return KERDOCK_ERR_INVALID_ARG;
  if (q > 65535 * int64_t(64)) return KERDOCK_ERR_UNSUPPORTED;  // GEMM grid rows
  *lay = shared_layout(p, q);
  if (ws == nullptr || ws_bytes < lay->total) return KERDOCK_ERR_CAPACITY;
  if (reinterpret_cast<uintptr_t>(ws) & 255) return KERDOCK_ERR_ALIGNMENT;
  return KERDOCK_OK;
}

}  // namespace
}  // namespace kd

extern "C" int kerdock_apply_shared(kerdock_plan_t plan, const float* X_dev, int64_t q,
                                    int64_t ldx, float eps, uint64_t seed, int32_t flags,
                                    int32_t* out_idx, float* out_val, int32_t* out_count,
                                    void* ws, size_t ws_bytes) {
  if (plan == nullptr || q < 0) return KERDOCK_ERR_INVALID_ARG;
  kd::Plan& p = plan->p;
  if (!p.bound) return KERDOCK_ERR_NOT_BOUND;
  if (!p.preprocessed) return KERDOCK_ERR_NOT_PREPROCESSED;
  if (q == 0) return KERDOCK_OK;
  if (out_idx == nullptr || out_val == nullptr || out_count == nullptr || flags < 0 ||
      flags > KERDOCK_FLAG_FULL_OUTPUT)
    return KERDOCK_ERR_INVALID_ARG;
  if (!(flags & KERDOCK_FLAG_FULL_OUTPUT) && !(eps > 0.0f)) return KERDOCK_ERR_INVALID_ARG;
  kd::SharedLayout lay;
  int rc = kd::shared_validate(p, X_dev, q, ldx, ws, ws_bytes, &lay);
  if (rc != KERDOCK_OK) return rc;
  char* base = static_cast<char*>(ws);
  float* scores = reinterpret_cast<float*>(base + lay.scores);
  rc = kd::shared_scores(p, X_dev, q, ldx, seed, base, lay, scores);
  if (rc != KERDOCK_OK) return rc;
  return kerdock_refine_scores(plan, X_dev, q, ldx, scores, p.S, eps, flags, out_idx, out_val,
                               out_count);
}

extern "C" int kerdock_apply_shared_scores(kerdock_plan_t plan, const float* X_dev, int64_t q,
                                           int64_t ldx, uint64_t seed, float* scores, void* ws,
                                           size_t ws_bytes) {
  if (plan == nullptr || q < 0) return KERDOCK_ERR_INVALID_ARG;
  kd::Plan& p = plan->p;
  if (!p.bound) return KERDOCK_ERR_NOT_BOUND;
  if (!p.preprocessed) return KERDOCK_ERR_NOT_PREPROCESSED;
  if (q == 0) return KERDOCK_OK;
  if (scores == nullptr) return KERDOCK_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(scores) & 15) return KERDOCK_ERR_ALIGNMENT;
  kd::SharedLayout lay;
  int rc = kd::shared_validate(p, X_dev, q, ldx, ws, ws_bytes, &lay);
  if (rc != KERDOCK_OK) return rc;
  return kd::shared_scores(p, X_dev, q, ldx, seed, static_cast<char*>(ws), lay, scores);
}
