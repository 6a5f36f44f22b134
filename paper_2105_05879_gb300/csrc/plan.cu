// plan.cu -- C ABI entry points (plan life cycle, binding, status) and the
// Kerdock sign-table kernel.
//
// The sign table is step (i) of Lemma 6: for every Kerdock matrix M_b of
// Prop. 5 and every point p of F_2^k, the bit Q_{M_b}(p) that decides the
// diagonal entry (-1)^{Q(p)} of D_{M_b}.  It is built on the device, one CTA
// per field element b, straight from the finite-field construction.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "kerdock_internal.cuh"

namespace kd {
namespace {

// Irreducible polynomials for GF(2^f), f = k - 1 (bit j = coefficient of t^j).
__constant__ uint32_t c_field_poly[kMaxLogD] = {0, 0x3, 0, 0xB, 0, 0x25, 0, 0x83, 0, 0x211, 0, 0x805};

// a * t in GF(2^f): shift, then fold the overflow back with the polynomial.
__device__ __forceinline__ uint32_t gf_xtime(uint32_t a, int f, uint32_t poly) {
  a <<= 1;
  return (a >> f) & 1u ? a ^ poly : a;
}

// Product by repeated doubling (a * b = sum_j b_j a t^j).
__device__ uint32_t gf_mul(uint32_t a, uint32_t b, int f, uint32_t poly) {
  uint32_t r = 0;
  for (int j = 0; j < f; ++j) {
    if ((b >> j) & 1u) r ^= a;
    a = gf_xtime(a, f, poly);
  }
  return r;
}

// The trace is F_2-linear, so tr(z) = parity(z & T) with T_j = tr(t^j); T is
// computed once per CTA from the definition tr(z) = sum_i z^(2^i).
__device__ uint32_t trace_mask(int f, uint32_t poly) {
  uint32_t T = 0;
  for (int j = 0; j < f; ++j) {
    uint32_t z = 1u << j, acc = 0;
    for (int i = 0; i < f; ++i) {
      acc ^= z;
      z = gf_mul(z, z, f, poly);
    }
    T |= (acc & 1u) << j;  // acc is 0 or 1 (the trace lands in F_2)
  }
  return T;
}

// One CTA per field element b.  Thread c < k forms L_b(B_c), the image of basis
// vector B_c, and from it column c of M_b: (M_b)_{a,c} = B_a . L_b(B_c) with
// (x,alpha).(y,beta) = tr(xy) + alpha*beta (Prop. 5).  Then Q_{M_b}(p) =
// sum_{a<c} M_ac p_a p_c = XOR over set bits a of p of parity(U_a & p), where
// U_a holds the entries of row a above the diagonal.
// Q_M(p) = XOR over set bits a of p of parity(U_a & p).
__device__ __forceinline__ uint32_t quad_form(const uint32_t* upper, int k, uint32_t p) {
  uint32_t q = 0;
  for (int a = 0; a < k; ++a)
    if ((p >> a) & 1u) q ^= __popc(upper[a] & p) & 1u;
  return q;
}

__global__ void signs_kernel(uint32_t* __restrict__ signs, uint32_t* __restrict__ tsigns, int k,
                             int64_t words_per_row, int64_t twords_per_row) {
  const int f = k - 1;
  const uint32_t poly = c_field_poly[f];
  const uint32_t b = blockIdx.x;
  const int64_t d = int64_t(1) << k;
  __shared__ uint32_t s_trace;
  __shared__ uint32_t s_col[kMaxLogD];
  __shared__ uint32_t s_upper[kMaxLogD];
  if (threadIdx.x == 0) s_trace = trace_mask(f, poly);
  __syncthreads();
  const uint32_t T = s_trace;
  if (threadIdx.x < k) {
    const int c = threadIdx.x;
    const uint32_t x = c < f ? (1u << c) : 0u;  // B_c = (t^c, 0) or (0, 1)
    const uint32_t alpha = c == f ? 1u : 0u;
    const uint32_t tr_bx = __popc(gf_mul(b, x, f, poly) & T) & 1u;
    uint32_t y = gf_mul(gf_mul(b, b, f, poly), x, f, poly);  // b^2 x
    if (tr_bx) y ^= b;                                        // + b tr(bx)
    if (alpha) y ^= b;                                        // + alpha b
    const uint32_t beta = tr_bx;
    uint32_t col = 0;
    for (int a = 0; a < f; ++a) {  // B_a = (t^a, 0): tr(t^a y)
      col |= (__popc(gf_mul(1u << a, y, f, poly) & T) & 1u) << a;
    }
    col |= beta << f;  // B_f = (0, 1): beta
    s_col[c] = col;
  }
  __syncthreads();
  if (threadIdx.x < k) {
    const int a = threadIdx.x;
    uint32_t U = 0;
    for (int c = a + 1; c < k; ++c) U |= ((s_col[c] >> a) & 1u) << c;
    s_upper[a] = U;
  }
  __syncthreads();
  // p-order table: each thread evaluates Q at one p, a warp ballot packs 32 bits.
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int64_t words = d >= 32 ? d / 32 : 1;
  for (int64_t w = warp; w < words; w += nwarps) {
    const int64_t p = w * 32 + lane;
    const uint32_t bits = __ballot_sync(0xffffffffu, p < d ? quad_form(s_upper, k, uint32_t(p)) : 0u);
    if (lane == 0) signs[int64_t(b) * words_per_row + w] = bits;
  }
  for (int64_t w = words + threadIdx.x; w < words_per_row; w += blockDim.x)
    signs[int64_t(b) * words_per_row + w] = 0u;  // row padding
  // Lane-transposed layout: word [g][L], bit t <-> p = 32 (32 g + t) + L.
  for (int64_t i = warp; i < twords_per_row; i += nwarps) {
    const int64_t g = i >> 5, L = i & 31;
    const int64_t p = 32 * (32 * g + lane) + L;
    const uint32_t bits = __ballot_sync(0xffffffffu, p < d ? quad_form(s_upper, k, uint32_t(p)) : 0u);
    if (lane == 0) tsigns[int64_t(b) * twords_per_row + i] = bits;
  }
}

// Failure-path check: wait, with a poll limit, on an mbarrier phase that no
// thread ever completes; give up, record a timeout in the status word and
// return -- the same bounded-wait-and-report path every kernel wait uses.
__global__ void wait_timeout_kernel(uint32_t* status, uint32_t max_polls) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    bool done = false;
    for (uint32_t it = 0; it < max_polls && !done; ++it) done = mbar_try_wait(&bar, 0);
    if (!done) set_status(status, kStatusTimeout);
  }
}

}  // namespace

int launch_signs(const Plan& p) {
  KD_CUDA_TRY(cudaMemsetAsync(p.table, 0, kStatusBytes, p.stream));
  signs_kernel<<<unsigned(p.d / 2), 256, 0, p.stream>>>(p.signs(), p.tsigns(), p.k,
                                                         p.sign_words, p.tsign_words);
  KD_CUDA_TRY(cudaGetLastError());
  return KERDOCK_OK;
}

}  // namespace kd

using kd::Plan;

extern "C" {

int kerdock_version(void) { return 100; }

const char* kerdock_strerror(int code) {
  switch (code) {
    case KERDOCK_OK: return "ok";
    case KERDOCK_ERR_INVALID_ARG: return "invalid argument";
    case KERDOCK_ERR_UNSUPPORTED: return "unsupported size or configuration";
    case KERDOCK_ERR_NOT_BOUND: return "plan has no device buffers bound";
    case KERDOCK_ERR_NOT_PREPROCESSED: return "kerdock_apply called before kerdock_preprocess";
    case KERDOCK_ERR_CAPACITY: return "a caller-provided buffer is too small";
    case KERDOCK_ERR_CUDA: return "a CUDA runtime call failed";
    case KERDOCK_ERR_DEVICE_TIMEOUT: return "a bounded device-side wait timed out";
    case KERDOCK_ERR_ALIGNMENT: return "a device pointer is not suitably aligned";
    default: return "unknown error";
  }
}

int kerdock_plan_create(kerdock_plan_t* plan, int64_t m, int64_t n, int32_t dtype, int32_t J,
                        int32_t K, int32_t S) {
  if (plan == nullptr) return KERDOCK_ERR_INVALID_ARG;
  *plan = nullptr;
  if (m < 1 || n < 1 || J < 1 || K < 1 || S < 1) return KERDOCK_ERR_INVALID_ARG;
  if (dtype != KERDOCK_F32 && dtype != KERDOCK_BF16) return KERDOCK_ERR_INVALID_ARG;
  if (m > 4096 || n > 4096 || K > kd::kMaxK) return KERDOCK_ERR_UNSUPPORTED;
  if (int64_t(J) * K > kd::kMaxN) return KERDOCK_ERR_UNSUPPORTED;
  auto* h = new (std::nothrow) kerdock_plan_s();
  if (h == nullptr) return KERDOCK_ERR_INVALID_ARG;
  Plan& p = h->p;
  p.m = m;
  p.n = n;
  p.k = 2;
  while ((int64_t(1) << p.k) < n) p.k += 2;  // smallest power of four >= n (Lemma 6)
  p.d = int64_t(1) << p.k;
  p.B = p.d / 2 + 1;
  p.L = p.d * p.B;
  p.ldr = (m + 7) / 8 * 8;
  p.dtype = dtype;
  p.J = J;
  p.K = K;
  p.S = int(S < m ? S : m);
  p.N = int64_t(J) * K;
  p.sign_words = p.d >= 128 ? p.d / 32 : 4;  // rows padded to 16 bytes (TMA copies)
  p.repr_bytes = size_t(p.B) * size_t(p.d) * size_t(p.ldr) * p.elem_bytes();
  p.tsign_words = p.d >= 1024 ? p.d / 32 : 32;
  p.table_bytes =
      kd::kStatusBytes + size_t(p.d / 2) * size_t(p.sign_words + p.tsign_words) * 4;
  *plan = h;
  return KERDOCK_OK;
}

int kerdock_plan_info(kerdock_plan_t plan, kerdock_plan_info_t* info) {
  if (plan == nullptr || info == nullptr) return KERDOCK_ERR_INVALID_ARG;
  const Plan& p = plan->p;
  std::memset(info, 0, sizeof(*info));
  info->m = p.m;
  info->n = p.n;
  info->k = p.k;
  info->dtype = p.dtype;
  info->d = p.d;
  info->num_bases = p.B;
  info->L = p.L;
  info->ldr = p.ldr;
  info->J = p.J;
  info->K = p.K;
  info->S = p.S;
  info->repr_bytes = p.repr_bytes;
  info->table_bytes = p.table_bytes;
  return KERDOCK_OK;
}

int kerdock_plan_bind(kerdock_plan_t plan, void* repr_dev, size_t repr_bytes, void* table_dev,
                      size_t table_bytes, void* stream) {
  if (plan == nullptr || repr_dev == nullptr || table_dev == nullptr)
    return KERDOCK_ERR_INVALID_ARG;
  Plan& p = plan->p;
  if (repr_bytes < p.repr_bytes || table_bytes < p.table_bytes) return KERDOCK_ERR_CAPACITY;
  if ((reinterpret_cast<uintptr_t>(repr_dev) & 255) || (reinterpret_cast<uintptr_t>(table_dev) & 255))
    return KERDOCK_ERR_ALIGNMENT;
  int dev = 0;
  KD_CUDA_TRY(cudaGetDevice(&dev));
  KD_CUDA_TRY(cudaDeviceGetAttribute(&p.num_sms, cudaDevAttrMultiProcessorCount, dev));
  p.device = dev;
  p.repr = repr_dev;
  p.table = table_dev;
  p.stream = static_cast<cudaStream_t>(stream);
  p.preprocessed = false;
  p.A = nullptr;
  const int rc = kd::launch_signs(p);
  if (rc != KERDOCK_OK) return rc;
  p.bound = true;
  return KERDOCK_OK;
}

int kerdock_set_stream(kerdock_plan_t plan, void* stream) {
  if (plan == nullptr) return KERDOCK_ERR_INVALID_ARG;
  plan->p.stream = static_cast<cudaStream_t>(stream);
  return KERDOCK_OK;
}

int kerdock_preprocess(kerdock_plan_t plan, const float* A_dev, int64_t lda) {
  if (plan == nullptr || A_dev == nullptr) return KERDOCK_ERR_INVALID_ARG;
  Plan& p = plan->p;
  if (!p.bound) return KERDOCK_ERR_NOT_BOUND;
  if (lda < p.n) return KERDOCK_ERR_INVALID_ARG;
  p.A = A_dev;
  p.lda = lda;
  const int rc = kd::launch_preprocess(p);
  if (rc != KERDOCK_OK) return rc;
  p.preprocessed = true;
  return KERDOCK_OK;
}

size_t kerdock_apply_workspace_bytes(kerdock_plan_t plan, int64_t q) {
  if (plan == nullptr || q < 0) return 0;
  return kd::apply_workspace_bytes(plan->p, q);
}

static int apply_common(kerdock_plan_t plan, const float* X, int64_t q, int64_t ldx, float eps,
                        uint64_t seed, int32_t flags, int32_t* out_idx, float* out_val,
                        int32_t* out_count, void* ws, size_t ws_bytes, float* mu_out,
                        int64_t* ells_out, float* coef_out) {
  if (plan == nullptr || q < 0) return KERDOCK_ERR_INVALID_ARG;
  Plan& p = plan->p;
  if (!p.bound) return KERDOCK_ERR_NOT_BOUND;
  if (!p.preprocessed) return KERDOCK_ERR_NOT_PREPROCESSED;
  if (q == 0) return KERDOCK_OK;
  if (X == nullptr || out_idx == nullptr || out_val == nullptr || out_count == nullptr)
    return KERDOCK_ERR_INVALID_ARG;
  if (ldx < p.n || flags < 0 || flags > KERDOCK_FLAG_FULL_OUTPUT) return KERDOCK_ERR_INVALID_ARG;
  if (!(flags & KERDOCK_FLAG_FULL_OUTPUT) && !(eps > 0.0f)) return KERDOCK_ERR_INVALID_ARG;
  if (q > (int64_t(1) << 31) / (p.S > 0 ? p.S : 1)) return KERDOCK_ERR_UNSUPPORTED;
  const size_t need = kd::apply_workspace_bytes(p, q);
  if (need > 0 && (ws == nullptr || ws_bytes < need)) return KERDOCK_ERR_CAPACITY;
  if (ws != nullptr && (reinterpret_cast<uintptr_t>(ws) & 255)) return KERDOCK_ERR_ALIGNMENT;
  return kd::launch_apply(p, X, q, ldx, eps, seed, flags, out_idx, out_val, out_count, ws,
                          ws_bytes, mu_out, ells_out, coef_out);
}

int kerdock_apply(kerdock_plan_t plan, const float* X_dev, int64_t q, int64_t ldx, float eps,
                  uint64_t seed, int32_t flags, int32_t* out_idx, float* out_val,
                  int32_t* out_count, void* ws_dev, size_t ws_bytes) {
  return apply_common(plan, X_dev, q, ldx, eps, seed, flags, out_idx, out_val, out_count, ws_dev,
                      ws_bytes, nullptr, nullptr, nullptr);
}

int kerdock_apply_debug(kerdock_plan_t plan, const float* X_dev, int64_t q, int64_t ldx,
                        float eps, uint64_t seed, int32_t flags, int32_t* out_idx,
                        float* out_val, int32_t* out_count, void* ws_dev, size_t ws_bytes,
                        float* mu_out, int64_t* ells_out, float* coef_out) {
  return apply_common(plan, X_dev, q, ldx, eps, seed, flags, out_idx, out_val, out_count, ws_dev,
                      ws_bytes, mu_out, ells_out, coef_out);
}

int kerdock_apply_noalloc(kerdock_plan_t plan, const float* X_dev, int64_t q, int64_t ldx,
                          float eps, uint64_t seed, int32_t flags, int32_t* out_idx,
                          float* out_val, int32_t* out_count) {
  if (plan == nullptr || q < 0) return KERDOCK_ERR_INVALID_ARG;
  Plan& p = plan->p;
  if (!p.bound) return KERDOCK_ERR_NOT_BOUND;
  if (!p.preprocessed) return KERDOCK_ERR_NOT_PREPROCESSED;
  if (q == 0) return KERDOCK_OK;
  if (X_dev == nullptr || out_idx == nullptr || out_val == nullptr || out_count == nullptr)
    return KERDOCK_ERR_INVALID_ARG;
  if (ldx < p.n || flags < 0 || flags > KERDOCK_FLAG_FULL_OUTPUT) return KERDOCK_ERR_INVALID_ARG;
  if (!(flags & KERDOCK_FLAG_FULL_OUTPUT) && !(eps > 0.0f)) return KERDOCK_ERR_INVALID_ARG;
  if (q > (int64_t(1) << 31) / (p.S > 0 ? p.S : 1)) return KERDOCK_ERR_UNSUPPORTED;
  // the scratch array is looked up for the current device: it must be the
  // device the plan's memory lives on
  int dev = 0;
  KD_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != p.device) return KERDOCK_ERR_INVALID_ARG;
  return kd::launch_apply_noalloc(p, X_dev, q, ldx, eps, seed, flags, out_idx, out_val,
                                  out_count);
}

int kerdock_sync(kerdock_plan_t plan) {
  if (plan == nullptr) return KERDOCK_ERR_INVALID_ARG;
  Plan& p = plan->p;
  if (!p.bound) return KERDOCK_ERR_NOT_BOUND;
  uint32_t status = 0;
  KD_CUDA_TRY(cudaMemcpyAsync(&status, p.status(), sizeof(status), cudaMemcpyDeviceToHost,
                              p.stream));
  KD_CUDA_TRY(cudaStreamSynchronize(p.stream));
  if (status != kd::kStatusOk) {
    KD_CUDA_TRY(cudaMemsetAsync(p.status(), 0, sizeof(uint32_t), p.stream));
    KD_CUDA_TRY(cudaStreamSynchronize(p.stream));
    return status == kd::kStatusTimeout ? KERDOCK_ERR_DEVICE_TIMEOUT : KERDOCK_ERR_INVALID_ARG;
  }
  return KERDOCK_OK;
}

int kerdock_debug_signs(kerdock_plan_t plan, uint32_t* host_out, size_t host_words) {
  if (plan == nullptr || host_out == nullptr) return KERDOCK_ERR_INVALID_ARG;
  Plan& p = plan->p;
  if (!p.bound) return KERDOCK_ERR_NOT_BOUND;
  const size_t words = size_t(p.d / 2) * size_t(p.sign_words);
  if (host_words < words) return KERDOCK_ERR_CAPACITY;
  KD_CUDA_TRY(cudaMemcpyAsync(host_out, p.signs(), words * 4, cudaMemcpyDeviceToHost, p.stream));
  KD_CUDA_TRY(cudaStreamSynchronize(p.stream));
  return KERDOCK_OK;
}

int kerdock_plan_clone(kerdock_plan_t* out, kerdock_plan_t src, int32_t J, int32_t K, int32_t S) {
  if (out == nullptr) return KERDOCK_ERR_INVALID_ARG;
  *out = nullptr;
  if (src == nullptr || J < 1 || K < 1 || S < 1) return KERDOCK_ERR_INVALID_ARG;
  if (K > kd::kMaxK || int64_t(J) * K > kd::kMaxN) return KERDOCK_ERR_UNSUPPORTED;
  auto* h = new (std::nothrow) kerdock_plan_s();
  if (h == nullptr) return KERDOCK_ERR_INVALID_ARG;
  h->p = src->p;  // shares the bound memory, stream, A and preprocessed state
  h->p.J = J;
  h->p.K = K;
  h->p.S = int(S < h->p.m ? S : h->p.m);
  h->p.N = int64_t(J) * K;
  h->p.tuning = kd::Tuning{};
  *out = h;
  return KERDOCK_OK;
}

int kerdock_debug_wait_timeout(kerdock_plan_t plan, int32_t max_polls) {
  if (plan == nullptr || max_polls < 1) return KERDOCK_ERR_INVALID_ARG;
  Plan& p = plan->p;
  if (!p.bound) return KERDOCK_ERR_NOT_BOUND;
  kd::wait_timeout_kernel<<<1, 32, 0, p.stream>>>(p.status(), uint32_t(max_polls));
  KD_CUDA_TRY(cudaGetLastError());
  return KERDOCK_OK;
}

int kerdock_debug_set_poll_limit(kerdock_plan_t plan, uint32_t max_polls) {
  if (plan == nullptr) return KERDOCK_ERR_INVALID_ARG;
  plan->p.poll_limit = max_polls == 0 ? kd::kDefaultPollLimit : max_polls;
  return KERDOCK_OK;
}

int kerdock_plan_destroy(kerdock_plan_t plan) {
  delete plan;
  return KERDOCK_OK;
}

}  // extern "C"

extern "C" int kerdock_theory_parameters(double a_row_norm_max, double eps, double delta,
                                         double eta, int64_t m, int32_t* J, int32_t* K) {
  if (J == nullptr || K == nullptr || !(a_row_norm_max > 0.0) || !(delta >= 0.0) ||
      !(eps > delta) || !(eta > 0.0) || !(eta <= 1.0) || m < 1)
    return KERDOCK_ERR_INVALID_ARG;
  const double gamma = 0.5 * (eps - delta);
  const double e = 2.718281828459045;  // Euler's number
  const double j = std::ceil(4.0 * e * e * a_row_norm_max * a_row_norm_max / (gamma * gamma));
  const double k = std::max(1.0, std::ceil(2.0 * std::log(double(m) / eta)));
  if (!(j < 2147483647.0)) return KERDOCK_ERR_UNSUPPORTED;
  *J = int32_t(j);
  *K = int32_t(k);
  if (k > double(kd::kMaxK) || j * k > double(kd::kMaxN)) return KERDOCK_ERR_UNSUPPORTED;
  return KERDOCK_OK;
}
