// check.cu -- FP64 checks of a device representation against A, on the GPU.
//
// Two identities of the paper pin the whole representation, not just samples
// of it, and are evaluated here in double precision:
//
//  * Reconstruction (Lemma 6 read backwards).  For a Kerdock basis b < d/2 the
//    stored slab is T_b = A Pi D_b W with W the +-1 Walsh matrix, and W W = d I,
//    so (1/d) (T_b W)[i][p] (-1)^{Q_b(p)} is A[i][p] for p < n and 0 for
//    p >= n.  For the identity basis, R[d/2][w][i] / sqrt(d) is A[i][w]
//    (0 for w >= n).  recon_kernel transforms every column i of a slab back
//    with an FP64 fast Walsh-Hadamard transform in shared memory and records
//    the largest deviation per basis.
//
//  * Tight frame (Prop. 2, through the design).  Every basis is orthonormal,
//    so sum_w s_{b,w} s_{b,w}^T = d I_n for each b, and the sampled rows
//    satisfy sum_{l in bases} R[l] <R[l], y> = (number of bases) d A A^T y for
//    any y in R^m; summed over all d/2 + 1 bases this is the tight-frame
//    identity sum_j B_j B_j^T = (d/2 + 1) I pushed through A.  frame_kernel
//    applies the left side to up to four probe vectors in one pass over the
//    representation; ref_kernel computes the right side from A.
#include "kerdock_internal.cuh"

namespace kd {
namespace {

constexpr int kCheckThreads = 512;
constexpr int kReconCols = 4;   // columns i per CTA: d = 4096 doubles x 4 = 128 KiB
constexpr int kMaxProbes = 4;
// Dynamic shared-memory caps, one per kernel for the whole process (captured
// graphs included), so each is set to the largest size the kernel takes
// (d, n <= 4096), never to one launch's size.
constexpr int kReconSmemCap = 4096 * kReconCols * int(sizeof(double));
constexpr int kRefSmemCap = 4096 * int(sizeof(double));

template <typename T>
__device__ __forceinline__ double load_rep(const T* p);
template <>
__device__ __forceinline__ double load_rep<float>(const float* p) {
  return double(*p);
}
template <>
__device__ __forceinline__ double load_rep<__nv_bfloat16>(const __nv_bfloat16* p) {
  return double(__bfloat162float(*p));
}

// Largest of non-negative doubles via their bit patterns (monotone as uint64).
__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(addr),
            static_cast<unsigned long long>(__double_as_longlong(v)));
}

struct ReconArgs {
  const void* R;
  int64_t ldr, m, n, d, b0;
  int k;
  const uint32_t* signs;  // p-order sign table, sign_words per basis
  int64_t sign_words;
  const float* A;
  int64_t lda;
  double* err;  // one per basis of the range
};

template <typename T>
__global__ void __launch_bounds__(kCheckThreads) recon_kernel(const ReconArgs a) {
  extern __shared__ __align__(16) double X[];  // [kReconCols][d]
  __shared__ double red[kCheckThreads / 32];
  const T* R = static_cast<const T*>(a.R);
  const int64_t d = a.d;
  const int64_t b = a.b0 + blockIdx.y;
  const int64_t i0 = int64_t(blockIdx.x) * kReconCols;
  const bool ident = b == d / 2;
  const T* slab = R + b * d * a.ldr;
  for (int64_t t = threadIdx.x; t < d * kReconCols; t += blockDim.x) {
    const int64_t w = t / kReconCols, c = t - w * kReconCols;
    X[c * d + w] = i0 + c < a.ldr ? load_rep<T>(slab + w * a.ldr + i0 + c) : 0.0;
  }
  __syncthreads();
  if (!ident) {
    // unnormalised FWHT along w of each column: log2(d) radix-2 passes
    const int64_t half = d / 2;
    for (int64_t h = 1; h < d; h <<= 1) {
      for (int64_t t = threadIdx.x; t < half * kReconCols; t += blockDim.x) {
        const int64_t c = t / half, u = t - c * half;
        const int64_t j = (u / h) * 2 * h + (u % h);
        double* col = X + c * d;
        const double x0 = col[j], x1 = col[j + h];
        col[j] = x0 + x1;
        col[j + h] = x0 - x1;
      }
      __syncthreads();
    }
  }
  const double scale = ident ? 1.0 / double(int64_t(1) << (a.k / 2)) : 1.0 / double(d);
  const uint32_t* srow = a.signs + (ident ? 0 : b) * a.sign_words;
  double worst = 0.0;
  for (int64_t t = threadIdx.x; t < d * kReconCols; t += blockDim.x) {
    const int64_t c = t / d, p = t - c * d;
    const int64_t i = i0 + c;
    if (i >= a.ldr) continue;
    double v = X[c * d + p] * scale;
    if (!ident && ((srow[p >> 5] >> (p & 31)) & 1u)) v = -v;
    // rows i in [m, ldr) of the layout are stored as 0
    const double want = (i < a.m && p < a.n) ? double(a.A[i * a.lda + p]) : 0.0;
    worst = fmax(worst, fabs(v - want));
  }
  for (int o = 16; o > 0; o >>= 1) worst = fmax(worst, __shfl_xor_sync(0xffffffffu, worst, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = worst;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < int(blockDim.x / 32); ++w) v = fmax(v, red[w]);
    atomic_max_nonneg(a.err + blockIdx.y, v);
  }
}

struct FrameArgs {
  const void* R;
  int64_t ldr, m, row0, rows;  // representation rows [row0, row0 + rows)
  const double* Y;             // P x m probes
  int P;
  double* out;                 // P x m, accumulated
};

// Persistent: CTA c takes a contiguous range of rows; per batch of 16 rows a
// warp forms the P products <R[l], y_p> of its row (FP64, warp reduction),
// then every thread adds R[l][i] <R[l], y_p> for its own columns i.
template <typename T, int U>
__global__ void __launch_bounds__(kCheckThreads, 1) frame_kernel(const FrameArgs a) {
  extern __shared__ __align__(16) double Ys[];  // [P][m]
  __shared__ double tdot[kCheckThreads / 32][kMaxProbes];
  const T* R = static_cast<const T*>(a.R);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int kWarps = kCheckThreads / 32;
  for (int64_t t = threadIdx.x; t < a.P * a.m; t += blockDim.x) Ys[t] = a.Y[t];
  double acc[U][kMaxProbes];
#pragma unroll
  for (int u = 0; u < U; ++u)
#pragma unroll
    for (int p = 0; p < kMaxProbes; ++p) acc[u][p] = 0.0;
  const int64_t per = (a.rows + gridDim.x - 1) / gridDim.x;
  const int64_t beg = a.row0 + int64_t(blockIdx.x) * per;
  int64_t end = beg + per;
  if (end > a.row0 + a.rows) end = a.row0 + a.rows;
  __syncthreads();
  for (int64_t r0 = beg; r0 < end; r0 += kWarps) {
    const int64_t l = r0 + warp;
    double part[kMaxProbes] = {0.0, 0.0, 0.0, 0.0};
    if (l < end) {
      const T* row = R + l * a.ldr;
      for (int64_t j = lane; j < a.m; j += 32) {
        const double v = load_rep<T>(row + j);
#pragma unroll
        for (int p = 0; p < kMaxProbes; ++p)
          if (p < a.P) part[p] = fma(v, Ys[p * a.m + j], part[p]);
      }
    }
#pragma unroll
    for (int p = 0; p < kMaxProbes; ++p)
      for (int o = 16; o > 0; o >>= 1) part[p] += __shfl_xor_sync(0xffffffffu, part[p], o);
    if (lane == 0)
#pragma unroll
      for (int p = 0; p < kMaxProbes; ++p) tdot[warp][p] = part[p];
    __syncthreads();
    const int nr = int(end - r0 < kWarps ? end - r0 : kWarps);
    for (int r = 0; r < nr; ++r) {
      const T* row = R + (r0 + r) * a.ldr;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t i = threadIdx.x + int64_t(u) * kCheckThreads;
        if (i < a.m) {
          const double v = load_rep<T>(row + i);
#pragma unroll
          for (int p = 0; p < kMaxProbes; ++p) acc[u][p] = fma(v, tdot[r][p], acc[u][p]);
        }
      }
    }
    __syncthreads();  // tdot is rewritten by the next batch
  }
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int64_t i = threadIdx.x + int64_t(u) * kCheckThreads;
    if (i < a.m) {
#pragma unroll
      for (int p = 0; p < kMaxProbes; ++p)
        if (p < a.P) atomicAdd(a.out + p * a.m + i, acc[u][p]);
    }
  }
}

// ref[p] = scale * A (A^T y_p) in FP64, one CTA per probe.
__global__ void __launch_bounds__(1024) ref_kernel(const float* A, int64_t lda, int64_t m,
                                                  int64_t n, const double* Y, double scale,
                                                  double* ref) {
  extern __shared__ __align__(16) double z[];  // [n]
  const int p = blockIdx.x;
  const double* y = Y + p * m;
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
    double s = 0.0;
    for (int64_t i = 0; i < m; ++i) s = fma(double(A[i * lda + j]), y[i], s);
    z[j] = s;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t i = warp; i < m; i += nw) {
    double s = 0.0;
    for (int64_t j = lane; j < n; j += 32) s = fma(double(A[i * lda + j]), z[j], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) ref[p * m + i] = scale * s;
  }
}

int check_range(const Plan& p, int64_t b0, int64_t nb) {
  if (!p.bound) return KERDOCK_ERR_NOT_BOUND;
  if (!p.preprocessed || p.A == nullptr) return KERDOCK_ERR_NOT_PREPROCESSED;
  if (b0 < 0 || nb < 1 || b0 + nb > p.B) return KERDOCK_ERR_INVALID_ARG;
  int dev = 0;
  KD_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != p.device) return KERDOCK_ERR_INVALID_ARG;
  return KERDOCK_OK;
}

template <typename T, int U>
int launch_frame(const FrameArgs& fa, const Plan& p, size_t smem) {
  auto kern = frame_kernel<T, U>;
  // the cap is per kernel and process-wide: the largest this instance takes
  // (kMaxProbes vectors of m <= U * kCheckThreads doubles), not this launch's
  constexpr int kCap = kMaxProbes * U * kCheckThreads * int(sizeof(double));
  if (smem > size_t(kCap)) return KERDOCK_ERR_UNSUPPORTED;
  KD_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kCap));
  kern<<<unsigned(p.num_sms), kCheckThreads, smem, p.stream>>>(fa);
  KD_CUDA_TRY(cudaGetLastError());
  return KERDOCK_OK;
}

}  // namespace
}  // namespace kd

using kd::Plan;

extern "C" int kerdock_check_reconstruction(kerdock_plan_t plan, int64_t b0, int64_t nb,
                                            double* err_dev) {
  if (plan == nullptr || err_dev == nullptr) return KERDOCK_ERR_INVALID_ARG;
  const Plan& p = plan->p;
  int rc = kd::check_range(p, b0, nb);
  if (rc != KERDOCK_OK) return rc;
  if (reinterpret_cast<uintptr_t>(err_dev) & 7) return KERDOCK_ERR_ALIGNMENT;
  if (nb > 65535) return KERDOCK_ERR_UNSUPPORTED;  // grid y
  KD_CUDA_TRY(cudaMemsetAsync(err_dev, 0, size_t(nb) * sizeof(double), p.stream));
  kd::ReconArgs a;
  a.R = p.repr;
  a.ldr = p.ldr;
  a.m = p.m;
  a.n = p.n;
  a.d = p.d;
  a.b0 = b0;
  a.k = p.k;
  a.signs = p.signs();
  a.sign_words = p.sign_words;
  a.A = p.A;
  a.lda = p.lda;
  a.err = err_dev;
  const size_t smem = size_t(p.d) * kd::kReconCols * sizeof(double);
  const dim3 grid(unsigned((p.ldr + kd::kReconCols - 1) / kd::kReconCols), unsigned(nb));
  if (p.dtype == KERDOCK_BF16) {
    KD_CUDA_TRY(cudaFuncSetAttribute(kd::recon_kernel<__nv_bfloat16>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, kd::kReconSmemCap));
    kd::recon_kernel<__nv_bfloat16><<<grid, kd::kCheckThreads, smem, p.stream>>>(a);
  } else {
    KD_CUDA_TRY(cudaFuncSetAttribute(kd::recon_kernel<float>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, kd::kReconSmemCap));
    kd::recon_kernel<float><<<grid, kd::kCheckThreads, smem, p.stream>>>(a);
  }
  KD_CUDA_TRY(cudaGetLastError());
  return KERDOCK_OK;
}

extern "C" int kerdock_check_tight_frame(kerdock_plan_t plan, const double* Y_dev, int32_t P,
                                         int64_t b0, int64_t nb, double* frame_dev,
                                         double* ref_dev) {
  if (plan == nullptr || Y_dev == nullptr || frame_dev == nullptr || ref_dev == nullptr)
    return KERDOCK_ERR_INVALID_ARG;
  if (P < 1 || P > kd::kMaxProbes) return KERDOCK_ERR_INVALID_ARG;
  const Plan& p = plan->p;
  int rc = kd::check_range(p, b0, nb);
  if (rc != KERDOCK_OK) return rc;
  if ((reinterpret_cast<uintptr_t>(Y_dev) | reinterpret_cast<uintptr_t>(frame_dev) |
       reinterpret_cast<uintptr_t>(ref_dev)) & 7)
    return KERDOCK_ERR_ALIGNMENT;
  KD_CUDA_TRY(cudaMemsetAsync(frame_dev, 0, size_t(P) * size_t(p.m) * sizeof(double), p.stream));
  kd::FrameArgs fa;
  fa.R = p.repr;
  fa.ldr = p.ldr;
  fa.m = p.m;
  fa.row0 = b0 * p.d;
  fa.rows = nb * p.d;
  fa.Y = Y_dev;
  fa.P = P;
  fa.out = frame_dev;
  const size_t smem = size_t(P) * size_t(p.m) * sizeof(double);
  const int64_t U = (p.m + kd::kCheckThreads - 1) / kd::kCheckThreads;  // m <= 4096: U <= 8
  const bool bf = p.dtype == KERDOCK_BF16;
  if (U <= 1)
    rc = bf ? kd::launch_frame<__nv_bfloat16, 1>(fa, p, smem) : kd::launch_frame<float, 1>(fa, p, smem);
  else if (U <= 2)
    rc = bf ? kd::launch_frame<__nv_bfloat16, 2>(fa, p, smem) : kd::launch_frame<float, 2>(fa, p, smem);
  else if (U <= 4)
    rc = bf ? kd::launch_frame<__nv_bfloat16, 4>(fa, p, smem) : kd::launch_frame<float, 4>(fa, p, smem);
  else
    rc = bf ? kd::launch_frame<__nv_bfloat16, 8>(fa, p, smem) : kd::launch_frame<float, 8>(fa, p, smem);
  if (rc != KERDOCK_OK) return rc;
  const size_t zsmem = size_t(p.n) * sizeof(double);
  KD_CUDA_TRY(cudaFuncSetAttribute(kd::ref_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   kd::kRefSmemCap));
  const double scale = double(nb) * double(p.d);
  kd::ref_kernel<<<unsigned(P), 1024, zsmem, p.stream>>>(p.A, p.lda, p.m, p.n, Y_dev, scale,
                                                         ref_dev);
  KD_CUDA_TRY(cudaGetLastError());
  return KERDOCK_OK;
}
