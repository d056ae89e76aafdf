// nmfa_api.cu -- the C ABI of libnmfa.so (declared in include/nmfa.h): argument
// checking, device copies of (h, J) in the storage each path needs, the per-handle
// scratch workspace, run orchestration on the caller's stream, and error codes.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "nmfa_internal.h"

namespace nmfa {

std::atomic<uint64_t> g_launches{0};

static thread_local std::string t_last_error;

int set_error(int code, const std::string& msg) {
  t_last_error = msg;
  return code;
}

int cuda_error(cudaError_t e, const char* where) {
  if (e == cudaSuccess) return NMFA_OK;
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return set_error(NMFA_ENOMEM, std::string(where) + ": " + cudaGetErrorString(e));
  }
  return set_error(NMFA_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

namespace {
struct PoolState {
  std::mutex mu;
  cudaStream_t alloc_stream[128] = {};
  cudaStream_t free_stream[128] = {};
};
PoolState& pool_state() {
  static PoolState s;
  return s;
}
// The current device's allocation stream (free = false) or release stream (true).
// Allocations and releases use separate streams: a release waits for the run that
// last used the buffer, and an allocation synchronises its own stream, so sharing
// one stream would make allocations wait for other runs.  The pool still hands a
// released block to a later allocation on the other stream once the release has
// executed.  The first call on a device also tells its default pool to keep freed
// memory and never to make an allocation wait for a pending release.
cudaStream_t pool_stream(bool free) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return nullptr;
  PoolState& ps = pool_state();
  std::lock_guard<std::mutex> g(ps.mu);
  if (ps.alloc_stream[dev] == nullptr) {
    cudaMemPool_t pool = nullptr;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t keep = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
      // never make an allocation wait for a pending release (it would wait for the
      // run the release waits for); reuse released blocks once they are free
      int no = 0;
      cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowInternalDependencies, &no);
    }
    cudaStream_t a = nullptr, f = nullptr;
    if (cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
    if (cudaStreamCreateWithFlags(&f, cudaStreamNonBlocking) != cudaSuccess) {
      cudaStreamDestroy(a);
      return nullptr;
    }
    ps.alloc_stream[dev] = a;
    ps.free_stream[dev] = f;
  }
  return free ? ps.free_stream[dev] : ps.alloc_stream[dev];
}
}  // namespace

int pool_alloc(void** p, size_t bytes) {
  *p = nullptr;
  cudaStream_t st = pool_stream(false);
  if (st == nullptr) return set_error(NMFA_ECUDA, "no allocation stream on this device");
  cudaError_t e = cudaMallocAsync(p, std::max<size_t>(bytes, 16), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    if (*p) cudaFreeAsync(*p, st);
    *p = nullptr;
    return cuda_error(e, "device allocation");
  }
  return NMFA_OK;
}

void pool_free(void* p, cudaEvent_t after) {
  if (p == nullptr) return;
  cudaStream_t st = pool_stream(true);
  if (st == nullptr) return;
  if (after != nullptr) cudaStreamWaitEvent(st, after, 0);
  cudaFreeAsync(p, st);
}

}  // namespace nmfa

using namespace nmfa;

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct nmfa_problem {
  int32_t n = 0;
  int32_t precision = 0;
  bool csr = false;
  bool integer_valued = false;
  bool int8_ok = false;  // integer problem with |J| <= 127: int8 energy copy
  // integer problem with max_i (sum_j |J_ij| + 2 |h_i|) < 2^24: the tensor kernel
  // forms the energies exactly in its own epilogue
  bool energy_exact = false;
  int32_t nnz = 0;
  int32_t n_pad = 0;
  int device = 0;
  // device copies
  double* J64 = nullptr;
  double* h64 = nullptr;
  double* d64 = nullptr;
  float* inv_d32 = nullptr;
  float* h32 = nullptr;
  float* J32 = nullptr;
  void* Jq = nullptr;      // bf16 / e4m3 padded (e4m3: groups of four as k0, k2, k1, k3)
  int8_t* J8 = nullptr;    // energy copy, rows padded to 16 bytes
  int32_t* row_ptr = nullptr;
  int32_t* col = nullptr;
  double* val64 = nullptr;
  float* val32 = nullptr;
  int8_t* val8 = nullptr;
  bool val_is_int8 = false;
  int64_t device_bytes = 0;
  std::vector<void*> allocations;
  // scratch
  DevBuf ws;              // kernel scratch (tensor path)
  DevBuf io;              // host-API staging: T, signs, energies
  DevBuf sign_scratch;    // signs when the caller does not want them
  int32_t* status = nullptr;
  cudaStream_t own_stream = nullptr;
  cudaEvent_t done = nullptr;
  cudaEvent_t prof0 = nullptr, prof1 = nullptr;
  bool profiling = false;
  bool prof_valid = false;
  int replicas_per_cta = 0;  // CUDA-core paths: 0 = automatic
  int32_t withhold_step = -1;  // nmfa_debug_withhold_arrival
  std::mutex mu;
};

namespace {

int dev_alloc(nmfa_problem* p, void** out, size_t bytes) {
  *out = nullptr;
  if (bytes == 0) bytes = 16;
  const int rc = pool_alloc(out, bytes);
  if (rc) return rc;
  p->allocations.push_back(*out);
  p->device_bytes += static_cast<int64_t>(bytes);
  return NMFA_OK;
}

template <typename T>
int dev_alloc_t(nmfa_problem* p, T** out, size_t count) {
  void* v = nullptr;
  int rc = dev_alloc(p, &v, count * sizeof(T));
  *out = static_cast<T*>(v);
  return rc;
}

// Grows a scratch buffer; the old one is released once `after` (the completion of
// the last run that may still use it, or nullptr) has completed.
int ensure_buf(DevBuf& b, size_t bytes, cudaEvent_t after = nullptr) {
  if (b.bytes >= bytes && b.p != nullptr) return NMFA_OK;
  if (b.p != nullptr) {
    pool_free(b.p, after);
    b.p = nullptr;
    b.bytes = 0;
  }
  const int rc = pool_alloc(&b.p, std::max<size_t>(bytes, 256));
  if (rc) return rc;
  b.bytes = std::max<size_t>(bytes, 256);
  return NMFA_OK;
}

bool bf16_exact(double v) {
  const float f = static_cast<float>(v);
  if (static_cast<double>(f) != v) return false;
  uint32_t bits;
  std::memcpy(&bits, &f, 4);
  return (bits & 0xFFFFu) == 0u;
}

// Exactly representable in FP8 E4M3 (bias 7, 3 mantissa bits, largest finite
// 448, subnormals k * 2^-9 for k = 1..7): |v| = m * 2^e with a 3-bit fraction.
bool e4m3_exact(double v) {
  if (v == 0.0) return true;
  const double a = std::fabs(v);
  if (!(a <= 448.0)) return false;
  int e = 0;
  const double fr = std::frexp(a, &e);  // a = fr * 2^e, fr in [0.5, 1)
  const int exp_unbiased = e - 1;       // a = (2 fr) * 2^(e-1), 2 fr in [1, 2)
  if (exp_unbiased < -6) {              // subnormal range: multiples of 2^-9
    const double k = std::ldexp(a, 9);
    return k == std::floor(k) && k >= 1.0 && k <= 7.0;
  }
  const double mant8 = (2.0 * fr - 1.0) * 8.0;  // exact in binary64
  return mant8 == std::floor(mant8);
}

// Host-side scan of a dense problem at creation: finiteness, zero diagonal,
// symmetry, integrality, the int8/BF16/E4M3 storage checks and the largest
// sum_j |J_ij| + 2 |h_i|.  Rows go in blocks of 32 to up to 16 threads; the symmetry
// check compares 32 x 32 tiles with their transposes, so that both reads stay in
// cache.  Errors are reported by kind in a fixed order (non-finite, diagonal,
// symmetry), not by position.
struct DenseScan {
  bool finite = true, diag_zero = true, symmetric = true;
  bool integer = true, int8_ok = true, bf16_ok = true, e4m3_ok = true;
  double max_row = 0.0;
};

void scan_rows(int32_t n, const double* h, const double* J, bool want_bf16, bool want_e4m3, int first_block,
               int stride, DenseScan* out) {
  constexpr int kB = 32;
  DenseScan r;
  const int64_t ln = n;
  for (int32_t ib = first_block * kB; ib < n; ib += stride * kB) {
    const int32_t ie = std::min(n, ib + kB);
    for (int32_t i = ib; i < ie; ++i) {
      double row = 0.0;
      if (h != nullptr) {
        const double hv = h[i];
        if (!std::isfinite(hv)) r.finite = false;
        if (hv != std::nearbyint(hv) || std::fabs(hv) >= 2147483648.0) r.integer = false;
        row = 2.0 * std::fabs(hv);
      }
      if (J[i * ln + i] != 0.0) r.diag_zero = false;
      const double* Ji = J + i * ln;
      for (int32_t j = 0; j < n; ++j) {
        const double v = Ji[j];
        const double a = std::fabs(v);
        if (!std::isfinite(v)) r.finite = false;
        if (v != std::nearbyint(v) || a >= 2147483648.0) r.integer = false;
        if (a > 127.0) r.int8_ok = false;
        row += a;
        // integers up to 16 in magnitude are exact in both BF16 and E4M3
        if (!(a <= 16.0 && v == std::nearbyint(v))) {
          if (want_bf16 && r.bf16_ok && !bf16_exact(v)) r.bf16_ok = false;
          if (want_e4m3 && r.e4m3_ok && !e4m3_exact(v)) r.e4m3_ok = false;
        }
      }
      r.max_row = std::max(r.max_row, row);
    }
    // symmetry: tiles (ib, jb) with jb >= ib against their transposes
    for (int32_t jb = ib; jb < n && r.symmetric; jb += kB) {
      const int32_t je = std::min(n, jb + kB);
      for (int32_t i = ib; i < ie; ++i)
        for (int32_t j = std::max(jb, i + 1); j < je; ++j)
          if (J[i * ln + j] != J[j * ln + i]) r.symmetric = false;
    }
  }
  *out = r;
}

DenseScan scan_dense(int32_t n, const double* h, const double* J, int32_t precision) {
  const bool want_bf16 = precision == NMFA_BF16, want_e4m3 = precision == NMFA_BF16_FP8J;
  int threads = 1;
  if (n >= 1024) {
    const unsigned hc = std::thread::hardware_concurrency();
    threads = static_cast<int>(std::min<unsigned>(16u, hc == 0 ? 1u : hc));
  }
  std::vector<DenseScan> parts(threads);
  if (threads == 1) {
    scan_rows(n, h, J, want_bf16, want_e4m3, 0, 1, &parts[0]);
  } else {
    std::vector<std::thread> pool;
    for (int t = 0; t < threads; ++t) pool.emplace_back(scan_rows, n, h, J, want_bf16, want_e4m3, t, threads, &parts[t]);
    for (auto& th : pool) th.join();
  }
  DenseScan r;
  for (const DenseScan& q : parts) {
    r.finite = r.finite && q.finite;
    r.diag_zero = r.diag_zero && q.diag_zero;
    r.symmetric = r.symmetric && q.symmetric;
    r.integer = r.integer && q.integer;
    r.int8_ok = r.int8_ok && q.int8_ok;
    r.bf16_ok = r.bf16_ok && q.bf16_ok;
    r.e4m3_ok = r.e4m3_ok && q.e4m3_ok;
    r.max_row = std::max(r.max_row, q.max_row);
  }
  return r;
}

// Host-built device copies of a tensor-path problem with integer |J_ij| <= 127 and
// integer |h_i| <= 2^20: every term of d_i^2 = h_i^2 + sum_j J_ij^2 is an integer
// and the sum stays below 2^53, so d_i computed here is bit-identical to the device
// kernel's (exact sum, correctly rounded square root), and the BF16 / E4M3 / int8
// copies are exact conversions.  Building them on the host avoids a binary64 device
// copy of J (8 n^2 bytes) and the device-wide synchronisation of freeing it, which
// otherwise stalls problem creation behind running kernels.
struct HostCompact {
  std::vector<double> d64;       // n
  std::vector<float> inv_d32;    // n_pad, 0 where d_i = 0 and in the padding
  std::vector<float> h32;        // n_pad, 0 in the padding
  std::vector<uint8_t> Jq;       // n_pad x n_pad BF16 or E4M3, zero-padded
  std::vector<int8_t> J8;        // n x ld8, rows padded with zeros
  int64_t ld8 = 0;
};

// v exactly representable in E4M3 (so also in binary32): the E4M3 fields are read off
// the binary32 pattern (exponent rebiased from 127 to 7, the top 3 fraction bits);
// below 2^-6 the value is k 2^-9 with k = 1..7 stored as the subnormal fraction.
uint8_t e4m3_bits(double v) {
  const float f = static_cast<float>(v);
  uint32_t b;
  std::memcpy(&b, &f, 4);
  const uint8_t sign = static_cast<uint8_t>((b >> 24) & 0x80u);
  if ((b & 0x7FFFFFFFu) == 0u) return sign;
  const int e = static_cast<int>((b >> 23) & 0xFFu) - 127;
  if (e >= -6) return static_cast<uint8_t>(sign | ((e + 7) << 3) | ((b >> 20) & 7u));
  return static_cast<uint8_t>(sign | static_cast<int>(std::fabs(f) * 512.0f));
}

uint16_t bf16_bits(double v) {  // v exactly representable in BF16
  const float f = static_cast<float>(v);
  uint32_t b;
  std::memcpy(&b, &f, 4);
  return static_cast<uint16_t>(b >> 16);
}

void compact_rows(int32_t n, int32_t n_pad, const double* h, const double* J, bool fp8, int first_block, int stride,
                  HostCompact* hc) {
  constexpr int kB = 32;
  const int64_t ln = n, lp = n_pad;
  for (int32_t ib = first_block * kB; ib < n; ib += stride * kB) {
    const int32_t ie = std::min(n, ib + kB);
    for (int32_t i = ib; i < ie; ++i) {
      const double* Ji = J + i * ln;
      double sq = 0.0;
      for (int32_t j = 0; j < n; ++j) {
        const double v = Ji[j];
        sq += v * v;
        hc->J8[i * hc->ld8 + j] = static_cast<int8_t>(v);
        if (fp8) {
          // groups of four in the order (k0, k2, k1, k3), as the tensor kernel reads them
          hc->Jq[i * lp + ((j & ~3) | ((j & 1) << 1) | ((j >> 1) & 1))] = e4m3_bits(v);
        } else {
          const uint16_t b = bf16_bits(v);
          std::memcpy(&hc->Jq[2 * (i * lp + j)], &b, 2);
        }
      }
      const double hv = h != nullptr ? h[i] : 0.0;
      const double d = std::sqrt(hv * hv + sq);
      hc->d64[i] = d;
      hc->inv_d32[i] = d > 0.0 ? static_cast<float>(1.0 / d) : 0.0f;
      hc->h32[i] = static_cast<float>(hv);
    }
  }
}

void build_compact(int32_t n, int32_t n_pad, const double* h, const double* J, bool fp8, HostCompact* hc) {
  hc->ld8 = (n + 15) / 16 * 16;
  hc->d64.assign(n, 0.0);
  hc->inv_d32.assign(std::max(n, n_pad), 0.0f);
  hc->h32.assign(std::max(n, n_pad), 0.0f);
  hc->Jq.assign(static_cast<size_t>(n_pad) * n_pad * (fp8 ? 1 : 2), 0);
  hc->J8.assign(static_cast<size_t>(n) * hc->ld8, 0);
  int threads = 1;
  if (n >= 1024) {
    const unsigned c = std::thread::hardware_concurrency();
    threads = static_cast<int>(std::min<unsigned>(16u, c == 0 ? 1u : c));
  }
  if (threads == 1) {
    compact_rows(n, n_pad, h, J, fp8, 0, 1, hc);
    return;
  }
  std::vector<std::thread> pool;
  for (int t = 0; t < threads; ++t) pool.emplace_back(compact_rows, n, n_pad, h, J, fp8, t, threads, hc);
  for (auto& th : pool) th.join();
}

int validate_common(int32_t n, int32_t precision) {
  if (n < 1 || n > 65536) return set_error(NMFA_EINVAL, "n must be in [1, 65536]");
  if (precision < NMFA_FP64 || precision > NMFA_BF16_FP8J)
    return set_error(NMFA_EINVAL, "unknown precision");
  return NMFA_OK;
}

int check_device() {
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess || count == 0) {
    cudaGetLastError();
    return set_error(NMFA_ECUDA, "no CUDA device available");
  }
  return NMFA_OK;
}

int finish_create(nmfa_problem* p, const double* h, const HostCompact* hc = nullptr) {
  int rc;
  if ((rc = cuda_error(cudaGetDevice(&p->device), "cudaGetDevice"))) return rc;
  if ((rc = cuda_error(cudaStreamCreateWithFlags(&p->own_stream, cudaStreamNonBlocking), "stream")))
    return rc;
  if ((rc = cuda_error(cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming), "event")))
    return rc;
  if ((rc = cuda_error(cudaEventCreate(&p->prof0), "event"))) return rc;
  if ((rc = cuda_error(cudaEventCreate(&p->prof1), "event"))) return rc;
  if ((rc = dev_alloc_t(p, &p->status, 4))) return rc;
  cudaStream_t st = p->own_stream;
  const int n = p->n;
  if ((rc = dev_alloc_t(p, &p->d64, n))) return rc;
  if ((rc = dev_alloc_t(p, &p->inv_d32, std::max(n, p->n_pad)))) return rc;
  if ((rc = dev_alloc_t(p, &p->h64, n))) return rc;
  if (h != nullptr) {
    if ((rc = cuda_error(cudaMemcpyAsync(p->h64, h, sizeof(double) * n, cudaMemcpyHostToDevice, st), "h upload")))
      return rc;
  } else {
    if ((rc = cuda_error(cudaMemsetAsync(p->h64, 0, sizeof(double) * n, st), "h clear"))) return rc;
  }
  // h in binary32, zero-padded to n_pad for the tensor path's padded rows
  if ((rc = dev_alloc_t(p, &p->h32, std::max(n, p->n_pad)))) return rc;
  if (hc != nullptr) {
    // norms and binary32 copies built on the host (exact for these problems)
    const size_t np = std::max(n, p->n_pad);
    if ((rc = cuda_error(cudaMemcpyAsync(p->h32, hc->h32.data(), sizeof(float) * np, cudaMemcpyHostToDevice, st),
                         "h upload")) ||
        (rc = cuda_error(cudaMemcpyAsync(p->inv_d32, hc->inv_d32.data(), sizeof(float) * np, cudaMemcpyHostToDevice,
                                         st),
                         "norm upload")) ||
        (rc = cuda_error(cudaMemcpyAsync(p->d64, hc->d64.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st),
                         "norm upload")))
      return rc;
    if ((rc = cuda_error(cudaMemsetAsync(p->status, 0, 4, st), "status clear"))) return rc;
    return cuda_error(cudaStreamSynchronize(st), "create");
  }
  if ((rc = cuda_error(cudaMemsetAsync(p->h32, 0, sizeof(float) * std::max(n, p->n_pad), st), "h clear"))) return rc;
  if ((rc = cuda_error(cudaMemsetAsync(p->inv_d32, 0, sizeof(float) * std::max(n, p->n_pad), st), "norm clear")))
    return rc;
  if ((rc = launch_convert_vec(n, p->h64, p->h32, 0, st))) return rc;
  if (p->csr) {
    if ((rc = launch_row_norms_csr(n, p->row_ptr, p->val64, p->h64, p->d64, p->inv_d32, st))) return rc;
  } else {
    if ((rc = launch_row_norms_dense(n, p->J64, p->h64, p->d64, p->inv_d32, st))) return rc;
  }
  if ((rc = cuda_error(cudaMemsetAsync(p->status, 0, 4, st), "status clear"))) return rc;
  return cuda_error(cudaStreamSynchronize(st), "create");
}

void free_problem(nmfa_problem* p) {
  if (p == nullptr) return;
  if (p->done) cudaEventSynchronize(p->done);
  for (void* a : p->allocations) pool_free(a);
  pool_free(p->ws.p);
  pool_free(p->io.p);
  pool_free(p->sign_scratch.p);
  if (p->done) cudaEventDestroy(p->done);
  if (p->prof0) cudaEventDestroy(p->prof0);
  if (p->prof1) cudaEventDestroy(p->prof1);
  if (p->own_stream) cudaStreamDestroy(p->own_stream);
  delete p;
}

}  // namespace

static int nmfa_autotuned_bn(nmfa_problem* p, int32_t replicas);

extern "C" {

const char* nmfa_last_error(void) { return t_last_error.c_str(); }

const char* nmfa_version(void) { return "nmfa-gb300 0.1 (sm_103a)"; }

uint64_t nmfa_launch_count(void) { return g_launches.load(); }

int nmfa_create(int32_t n, const double* h, const double* J, int32_t precision, nmfa_problem** out) {
  if (out == nullptr) return set_error(NMFA_EINVAL, "out is NULL");
  *out = nullptr;
  int rc = validate_common(n, precision);
  if (rc) return rc;
  if (J == nullptr) return set_error(NMFA_EINVAL, "J is NULL");
  const DenseScan sc = scan_dense(n, h, J, precision);
  if (!sc.finite) return set_error(NMFA_EINVAL, "h or J has a non-finite entry");
  if (!sc.diag_zero) return set_error(NMFA_EDIAG, "J has a nonzero diagonal entry");
  if (!sc.symmetric) return set_error(NMFA_ENOTSYM, "J is not symmetric");
  const bool integer = sc.integer;
  const bool int8_ok = sc.int8_ok && integer && static_cast<int64_t>(n) * 127 < (1ll << 30);
  const double max_row = sc.max_row;
  if (precision == NMFA_BF16 && !sc.bf16_ok)
    return set_error(NMFA_EUNSUPPORTED, "J is not exactly representable in BF16");
  if (precision == NMFA_BF16_FP8J && !sc.e4m3_ok)
    return set_error(NMFA_EUNSUPPORTED, "J is not exactly representable in FP8 E4M3");
  if ((rc = check_device())) return rc;
  nmfa_problem* p = new nmfa_problem();
  p->n = n;
  p->precision = precision;
  p->integer_valued = integer;
  p->int8_ok = int8_ok;
  p->energy_exact = integer && max_row < 16777216.0;
  p->n_pad = (n + 127) / 128 * 128;
  cudaStream_t st = nullptr;
  auto fail = [&](int code) {
    std::string msg = t_last_error;
    free_problem(p);
    t_last_error = msg;
    return code;
  };
  // Tensor-path problems with |J_ij| <= 127 integers and small integer h are
  // prepared on the host (see HostCompact); the rest go through a binary64 device
  // copy of J.
  bool compact = (precision == NMFA_BF16 || precision == NMFA_BF16_FP8J) && int8_ok;
  if (compact && h != nullptr)
    for (int32_t i = 0; i < n && compact; ++i) compact = std::fabs(h[i]) <= 1048576.0;
  if (compact) {
    HostCompact hc;
    build_compact(n, p->n_pad, h, J, precision == NMFA_BF16_FP8J, &hc);
    if ((rc = finish_create(p, h, &hc))) return fail(rc);
    st = p->own_stream;
    void* q = nullptr;
    if ((rc = dev_alloc(p, &q, hc.Jq.size()))) return fail(rc);
    p->Jq = q;
    if ((rc = dev_alloc_t(p, &p->J8, hc.J8.size()))) return fail(rc);
    if ((rc = cuda_error(cudaMemcpyAsync(p->Jq, hc.Jq.data(), hc.Jq.size(), cudaMemcpyHostToDevice, st), "J upload")) ||
        (rc = cuda_error(cudaMemcpyAsync(p->J8, hc.J8.data(), hc.J8.size(), cudaMemcpyHostToDevice, st), "J upload")) ||
        (rc = cuda_error(cudaStreamSynchronize(st), "J upload")))
      return fail(rc);
    *out = p;
    return NMFA_OK;
  }
  if ((rc = dev_alloc_t(p, &p->J64, static_cast<size_t>(n) * n))) return fail(rc);
  if ((rc = cuda_error(cudaMemcpy(p->J64, J, sizeof(double) * n * static_cast<size_t>(n), cudaMemcpyHostToDevice), "J upload")))
    return fail(rc);
  if ((rc = finish_create(p, h))) return fail(rc);
  st = p->own_stream;
  if (precision == NMFA_FP32) {
    // n_pad x n_pad with zeros beyond n: the tiled kernel's tiles need no bounds checks
    if ((rc = dev_alloc_t(p, &p->J32, static_cast<size_t>(p->n_pad) * p->n_pad))) return fail(rc);
    if ((rc = launch_convert_dense(n, p->J64, p->J32, 0, p->n_pad, p->n_pad, st))) return fail(rc);
  } else if (precision == NMFA_BF16 || precision == NMFA_BF16_FP8J) {
    const size_t elem = precision == NMFA_BF16 ? 2 : 1;
    void* q = nullptr;
    if ((rc = dev_alloc(p, &q, elem * p->n_pad * static_cast<size_t>(p->n_pad)))) return fail(rc);
    p->Jq = q;
    if ((rc = launch_convert_dense(n, p->J64, p->Jq, precision == NMFA_BF16 ? 1 : 2, p->n_pad, p->n_pad, st)))
      return fail(rc);
  }
  if (int8_ok) {
    const int64_t ld8 = (n + 15) / 16 * 16;
    if ((rc = dev_alloc_t(p, &p->J8, static_cast<size_t>(n) * ld8))) return fail(rc);
    if ((rc = launch_convert_dense(n, p->J64, p->J8, 3, n, ld8, st))) return fail(rc);
  }
  if ((rc = cuda_error(cudaStreamSynchronize(st), "create conversions"))) return fail(rc);
  // Tensor-path problems with integer couplings keep only the compact copies: the
  // FP64 matrix served the row norms and is not read again (energies use int8).
  if ((precision == NMFA_BF16 || precision == NMFA_BF16_FP8J) && int8_ok) {
    auto it = std::find(p->allocations.begin(), p->allocations.end(), static_cast<void*>(p->J64));
    if (it != p->allocations.end()) {
      pool_free(p->J64);
      p->allocations.erase(it);
      p->device_bytes -= static_cast<int64_t>(sizeof(double)) * n * n;
      p->J64 = nullptr;
    }
  }
  *out = p;
  return NMFA_OK;
}

int nmfa_create_csr(int32_t n, const double* h, const int64_t* row_ptr, const int32_t* col,
                    const double* val, int32_t precision, nmfa_problem** out) {
  if (out == nullptr) return set_error(NMFA_EINVAL, "out is NULL");
  *out = nullptr;
  int rc = validate_common(n, precision);
  if (rc) return rc;
  if (precision != NMFA_FP32 && precision != NMFA_FP64)
    return set_error(NMFA_EUNSUPPORTED, "CSR input takes NMFA_FP32 or NMFA_FP64 only");
  if (row_ptr == nullptr) return set_error(NMFA_EINVAL, "row_ptr is NULL");
  if (row_ptr[0] != 0) return set_error(NMFA_EINVAL, "row_ptr[0] must be 0");
  const int64_t nnz = row_ptr[n];
  if (nnz < 0 || nnz > (1ll << 31) - 1) return set_error(NMFA_EINVAL, "bad nnz");
  if (nnz > 0 && (col == nullptr || val == nullptr)) return set_error(NMFA_EINVAL, "col/val is NULL");
  bool integer = true, int8_ok = true;
  for (int32_t i = 0; i < n; ++i) {
    if (row_ptr[i + 1] < row_ptr[i]) return set_error(NMFA_EINVAL, "row_ptr is not monotone");
    if (h != nullptr) {
      if (!std::isfinite(h[i])) return set_error(NMFA_EINVAL, "h has a non-finite entry");
      if (h[i] != std::nearbyint(h[i]) || std::fabs(h[i]) >= 2147483648.0) integer = false;
    }
    for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q) {
      const int32_t j = col[q];
      if (j < 0 || j >= n) return set_error(NMFA_EINVAL, "column index out of range");
      if (q > row_ptr[i] && col[q - 1] >= j) return set_error(NMFA_EINVAL, "columns must ascend within a row");
      if (j == i) return set_error(NMFA_EDIAG, "CSR has a diagonal entry");
      const double v = val[q];
      if (!std::isfinite(v)) return set_error(NMFA_EINVAL, "val has a non-finite entry");
      if (v != std::nearbyint(v) || std::fabs(v) >= 2147483648.0) integer = false;
      if (std::fabs(v) > 127.0) int8_ok = false;
      // symmetric: find (j, i) by binary search in row j
      const int32_t* b = col + row_ptr[j];
      const int32_t* e = col + row_ptr[j + 1];
      const int32_t* f = std::lower_bound(b, e, i);
      if (f == e || *f != i || val[row_ptr[j] + (f - b)] != v) return set_error(NMFA_ENOTSYM, "CSR J is not symmetric");
    }
  }
  if ((rc = check_device())) return rc;
  nmfa_problem* p = new nmfa_problem();
  p->n = n;
  p->precision = precision;
  p->csr = true;
  p->nnz = static_cast<int32_t>(nnz);
  p->integer_valued = integer;
  p->int8_ok = false;  // energies of CSR problems use the CSR form
  p->val_is_int8 = integer && int8_ok;
  p->n_pad = n;
  auto fail = [&](int code) {
    std::string msg = t_last_error;
    free_problem(p);
    t_last_error = msg;
    return code;
  };
  std::vector<int32_t> rp32(n + 1);
  for (int32_t i = 0; i <= n; ++i) rp32[i] = static_cast<int32_t>(row_ptr[i]);
  if ((rc = dev_alloc_t(p, &p->row_ptr, n + 1))) return fail(rc);
  if ((rc = dev_alloc_t(p, &p->col, std::max<int64_t>(nnz, 1)))) return fail(rc);
  if ((rc = dev_alloc_t(p, &p->val64, std::max<int64_t>(nnz, 1)))) return fail(rc);
  if ((rc = cuda_error(cudaMemcpy(p->row_ptr, rp32.data(), 4 * (n + 1), cudaMemcpyHostToDevice), "CSR upload")))
    return fail(rc);
  if (nnz > 0) {
    if ((rc = cuda_error(cudaMemcpy(p->col, col, 4 * nnz, cudaMemcpyHostToDevice), "CSR upload"))) return fail(rc);
    if ((rc = cuda_error(cudaMemcpy(p->val64, val, 8 * nnz, cudaMemcpyHostToDevice), "CSR upload"))) return fail(rc);
  }
  if ((rc = finish_create(p, h))) return fail(rc);
  cudaStream_t st = p->own_stream;
  if (precision == NMFA_FP32) {
    if (p->val_is_int8) {
      if ((rc = dev_alloc_t(p, &p->val8, std::max<int64_t>(nnz, 1)))) return fail(rc);
      if (nnz > 0 && (rc = launch_convert_vec(static_cast<int32_t>(nnz), p->val64, p->val8, 3, st))) return fail(rc);
    } else {
      if ((rc = dev_alloc_t(p, &p->val32, std::max<int64_t>(nnz, 1)))) return fail(rc);
      if (nnz > 0 && (rc = launch_convert_vec(static_cast<int32_t>(nnz), p->val64, p->val32, 0, st))) return fail(rc);
    }
  } else if (p->val_is_int8) {
    // FP64 path keeps FP64 values so that its sums match an FP64 evaluation.
    p->val_is_int8 = false;
  }
  if ((rc = cuda_error(cudaStreamSynchronize(st), "create conversions"))) return fail(rc);
  *out = p;
  return NMFA_OK;
}

void nmfa_destroy(nmfa_problem* p) { free_problem(p); }

int nmfa_problem_info(const nmfa_problem* p, int32_t* n, int32_t* precision, int32_t* integer_valued,
                      int64_t* device_bytes) {
  if (p == nullptr) return set_error(NMFA_EINVAL, "NULL handle");
  if (n) *n = p->n;
  if (precision) *precision = p->precision;
  if (integer_valued) *integer_valued = p->integer_valued ? 1 : 0;
  if (device_bytes) *device_bytes = p->device_bytes + static_cast<int64_t>(p->ws.bytes + p->io.bytes + p->sign_scratch.bytes);
  return NMFA_OK;
}

int nmfa_profile_enable(nmfa_problem* p, int32_t on) {
  if (p == nullptr) return set_error(NMFA_EINVAL, "NULL handle");
  p->profiling = on != 0;
  p->prof_valid = false;
  return NMFA_OK;
}

int nmfa_measure_alu_peaks(double* out, void* cuda_stream) {
  if (out == nullptr) return set_error(NMFA_EINVAL, "out is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  double r[3] = {0.0, 0.0, 0.0};
  for (int k = 0; k < 3; ++k) {
    const int rc = measure_alu_peak(k, st, &r[k]);
    if (rc) return rc;
  }
  for (int k = 0; k < 3; ++k) out[k] = r[k];
  return NMFA_OK;
}

int nmfa_last_kernel_ms(nmfa_problem* p, float* ms) {
  if (p == nullptr || ms == nullptr) return set_error(NMFA_EINVAL, "NULL argument");
  if (!p->prof_valid) return set_error(NMFA_EINVAL, "no profiled run");
  int rc = cuda_error(cudaEventSynchronize(p->prof1), "profile sync");
  if (rc) return rc;
  return cuda_error(cudaEventElapsedTime(ms, p->prof0, p->prof1), "profile elapsed");
}

int nmfa_sync(nmfa_problem* p) {
  if (p == nullptr) return set_error(NMFA_EINVAL, "NULL handle");
  int rc = cuda_error(cudaEventSynchronize(p->done), "sync");
  if (rc) return rc;
  int32_t st = 0;
  rc = cuda_error(cudaMemcpy(&st, p->status, 4, cudaMemcpyDeviceToHost), "status read");
  if (rc) return rc;
  if (st != kStatusOk) {
    cudaMemset(p->status, 0, 4);
    return set_error(NMFA_ETIMEOUT, "a bounded device-side wait gave up (status " + std::to_string(st) + ")");
  }
  return NMFA_OK;
}

static int run_impl(nmfa_problem* p, const double* T_dev, int32_t t_f, double sigma, double alpha,
                    int32_t replicas, uint64_t seed, uint32_t stream_id, int32_t noise_sign,
                    const double* s0_dev, double* s_out_dev, double* phi_out_dev, int8_t* signs_dev,
                    double* energy_dev, int64_t* energy_i64_dev, cudaStream_t st) {
  if (p == nullptr) return set_error(NMFA_EINVAL, "NULL handle");
  if (t_f < 0) return set_error(NMFA_EINVAL, "t_f must be >= 0");
  if (t_f > 0 && T_dev == nullptr) return set_error(NMFA_EINVAL, "T is NULL");
  if (!(sigma >= 0.0) || !std::isfinite(sigma)) return set_error(NMFA_EINVAL, "sigma must be >= 0");
  if (!(alpha > 0.0 && alpha <= 1.0)) return set_error(NMFA_EINVAL, "alpha must be in (0, 1]");
  if (replicas < 1) return set_error(NMFA_EINVAL, "replicas must be >= 1");
  if (noise_sign < -1 || noise_sign > 1) return set_error(NMFA_EINVAL, "noise_sign must be -1, 0 or 1");
  if (energy_i64_dev != nullptr && !p->integer_valued)
    return set_error(NMFA_EINVAL, "integer energies requested for a real-valued problem");
  if (static_cast<int64_t>(replicas) * p->n > (1ll << 40)) return set_error(NMFA_EINVAL, "replicas * n too large");
  int rc;
  if ((rc = cuda_error(cudaSetDevice(p->device), "cudaSetDevice"))) return rc;
  // Runs on one handle share its scratch: order this run after the previous one.
  if ((rc = cuda_error(cudaStreamWaitEvent(st, p->done, 0), "stream wait"))) return rc;
  if (signs_dev == nullptr) {
    if ((rc = ensure_buf(p->sign_scratch, static_cast<size_t>(replicas) * p->n, p->done))) return rc;
    signs_dev = static_cast<int8_t*>(p->sign_scratch.p);
  }
  RunParams rp{};
  rp.T = T_dev;
  rp.t_f = t_f;
  rp.sigma = sigma;
  rp.alpha = alpha;
  rp.replicas = replicas;
  rp.seed = seed;
  rp.stream_id = stream_id;
  rp.noise_sign = noise_sign;
  rp.s0 = s0_dev;
  rp.s_out = s_out_dev;
  rp.phi_out = phi_out_dev;
  rp.signs = signs_dev;
  rp.energy = energy_dev;
  rp.energy_i64 = energy_i64_dev;
  bool energy_fused = false;
  if (p->profiling && (rc = cuda_error(cudaEventRecord(p->prof0, st), "profile event"))) return rc;
  switch (p->precision) {
    case NMFA_FP64:
    case NMFA_FP32: {
      const bool f64 = p->precision == NMFA_FP64;
      if (p->csr) {
        CsrProblem pb{};
        pb.n = p->n;
        pb.nnz = p->nnz;
        pb.row_ptr = p->row_ptr;
        pb.col = p->col;
        pb.val_int8 = !f64 && p->val_is_int8;
        pb.val = f64 ? static_cast<const void*>(p->val64)
                     : (pb.val_int8 ? static_cast<const void*>(p->val8) : static_cast<const void*>(p->val32));
        pb.h = f64 ? static_cast<const void*>(p->h64) : static_cast<const void*>(p->h32);
        pb.d = p->d64;
        pb.inv_d32 = p->inv_d32;
        rc = launch_csr(f64, pb, rp, st, p->replicas_per_cta);
      } else {
        DenseSimtProblem pb{};
        pb.n = p->n;
        pb.J = f64 ? static_cast<const void*>(p->J64) : static_cast<const void*>(p->J32);
        pb.ldj = f64 ? p->n : p->n_pad;
        pb.h = f64 ? static_cast<const void*>(p->h64) : static_cast<const void*>(p->h32);
        pb.d = p->d64;
        pb.inv_d32 = p->inv_d32;
        if (!f64 && tiled_f32_preferred(p->n, replicas) && p->replicas_per_cta == 0) {
          if ((rc = ensure_buf(p->ws, static_cast<size_t>(tiled_f32_workspace_bytes(p->n, replicas)), p->done)))
            return rc;
          rc = launch_dense_tiled_f32(pb, rp, p->ws.p, p->status, p->withhold_step, st);
        } else {
          rc = launch_dense_simt(f64, pb, rp, st, p->replicas_per_cta);
        }
      }
      break;
    }
    default: {
      TcProblem pb{};
      pb.n = p->n;
      pb.n_pad = p->n_pad;
      pb.Jq = p->Jq;
      // FP8-stored couplings are read as stored: the kernel's converter warps expand
      // each staged E4M3 slice to BF16 in shared memory
      pb.fp8 = p->precision == NMFA_BF16_FP8J;
      pb.inv_d32 = p->inv_d32;
      pb.h32 = p->h32;
      pb.energy_exact = p->energy_exact;
      energy_fused = tc_fuses_energy(pb, rp);
      int64_t bytes = 0;
      if ((rc = tc_workspace_bytes(pb, replicas, &bytes))) return rc;
      if ((rc = ensure_buf(p->ws, static_cast<size_t>(bytes), p->done))) return rc;
      TcWorkspace ws{};
      ws.S16 = p->ws.p;
      ws.bytes = bytes;
      ws.status = p->status;
      rc = launch_tc(pb, rp, ws, st);
      break;
    }
  }
  if (rc) return rc;
  if (p->profiling) {
    if ((rc = cuda_error(cudaEventRecord(p->prof1, st), "profile event"))) return rc;
    p->prof_valid = true;
  }
  if (!energy_fused && (energy_dev != nullptr || energy_i64_dev != nullptr)) {
    EnergyProblem ep{};
    ep.n = p->n;
    ep.J8 = p->J8;
    ep.J64 = p->csr ? nullptr : p->J64;
    ep.row_ptr = p->csr ? p->row_ptr : nullptr;
    ep.col = p->col;
    ep.val64 = p->val64;
    ep.h = p->h64;
    ep.integer_valued = p->integer_valued;
    if ((rc = launch_energy(ep, signs_dev, replicas, energy_dev, energy_i64_dev, st))) return rc;
  }
  return cuda_error(cudaEventRecord(p->done, st), "event record");
}

int nmfa_run_device(nmfa_problem* p, const double* T_dev, int32_t t_f, double sigma, double alpha,
                    int32_t replicas, uint64_t seed, uint32_t stream_id, int8_t* signs_dev,
                    double* energy_dev, int64_t* energy_i64_dev, void* cuda_stream) {
  if (p == nullptr) return set_error(NMFA_EINVAL, "NULL handle");
  std::lock_guard<std::mutex> g(p->mu);
  return run_impl(p, T_dev, t_f, sigma, alpha, replicas, seed, stream_id, 1, nullptr, nullptr, nullptr,
                  signs_dev, energy_dev, energy_i64_dev, static_cast<cudaStream_t>(cuda_stream));
}

int nmfa_debug_run(nmfa_problem* p, const double* T_dev, int32_t t_f, double sigma, double alpha,
                   int32_t replicas, uint64_t seed, uint32_t stream_id, int32_t noise_sign,
                   const double* s0_dev, double* s_out_dev, double* phi_out_dev, int8_t* signs_dev,
                   double* energy_dev, int64_t* energy_i64_dev, void* cuda_stream) {
  if (p == nullptr) return set_error(NMFA_EINVAL, "NULL handle");
  std::lock_guard<std::mutex> g(p->mu);
  return run_impl(p, T_dev, t_f, sigma, alpha, replicas, seed, stream_id, noise_sign, s0_dev, s_out_dev,
                  phi_out_dev, signs_dev, energy_dev, energy_i64_dev, static_cast<cudaStream_t>(cuda_stream));
}

int nmfa_run(nmfa_problem* p, const double* T, int32_t t_f, double sigma, double alpha, int32_t replicas,
             uint64_t seed, uint32_t stream_id, int8_t* signs_out, double* energy_out, int64_t* energy_i64_out) {
  if (p == nullptr) return set_error(NMFA_EINVAL, "NULL handle");
  if (t_f < 0 || replicas < 1) return set_error(NMFA_EINVAL, "t_f must be >= 0 and replicas >= 1");
  if (t_f > 0 && T == nullptr) return set_error(NMFA_EINVAL, "T is NULL");
  for (int32_t t = 0; t < t_f; ++t)
    if (!(T[t] > 0.0) || !std::isfinite(T[t])) return set_error(NMFA_EINVAL, "every T_t must be finite and > 0");
  if (energy_i64_out != nullptr && !p->integer_valued)
    return set_error(NMFA_EINVAL, "integer energies requested for a real-valued problem");
  std::lock_guard<std::mutex> g(p->mu);
  const size_t signs_b = static_cast<size_t>(replicas) * p->n;
  const size_t off_T = 0;
  const size_t off_E = (sizeof(double) * std::max(t_f, 1) + 255) / 256 * 256;
  const size_t off_Ei = off_E + (sizeof(double) * replicas + 255) / 256 * 256;
  const size_t off_S = off_Ei + (sizeof(int64_t) * replicas + 255) / 256 * 256;
  int rc;
  if ((rc = cuda_error(cudaSetDevice(p->device), "cudaSetDevice"))) return rc;
  if ((rc = cuda_error(cudaEventSynchronize(p->done), "sync"))) return rc;
  if ((rc = ensure_buf(p->io, off_S + signs_b))) return rc;
  char* base = static_cast<char*>(p->io.p);
  double* T_dev = reinterpret_cast<double*>(base + off_T);
  double* E_dev = reinterpret_cast<double*>(base + off_E);
  int64_t* Ei_dev = reinterpret_cast<int64_t*>(base + off_Ei);
  int8_t* S_dev = reinterpret_cast<int8_t*>(base + off_S);
  cudaStream_t st = p->own_stream;
  if (t_f > 0 && (rc = cuda_error(cudaMemcpyAsync(T_dev, T, sizeof(double) * t_f, cudaMemcpyHostToDevice, st), "T upload")))
    return rc;
  rc = run_impl(p, T_dev, t_f, sigma, alpha, replicas, seed, stream_id, 1, nullptr, nullptr, nullptr, S_dev,
                energy_out ? E_dev : nullptr, energy_i64_out ? Ei_dev : nullptr, st);
  if (rc) return rc;
  if (signs_out && (rc = cuda_error(cudaMemcpyAsync(signs_out, S_dev, signs_b, cudaMemcpyDeviceToHost, st), "signs download")))
    return rc;
  if (energy_out && (rc = cuda_error(cudaMemcpyAsync(energy_out, E_dev, sizeof(double) * replicas, cudaMemcpyDeviceToHost, st), "energy download")))
    return rc;
  if (energy_i64_out && (rc = cuda_error(cudaMemcpyAsync(energy_i64_out, Ei_dev, sizeof(int64_t) * replicas, cudaMemcpyDeviceToHost, st), "energy download")))
    return rc;
  if ((rc = cuda_error(cudaStreamSynchronize(st), "run"))) return rc;
  int32_t status = 0;
  if ((rc = cuda_error(cudaMemcpy(&status, p->status, 4, cudaMemcpyDeviceToHost), "status read"))) return rc;
  if (status != kStatusOk) {
    cudaMemset(p->status, 0, 4);
    return set_error(NMFA_ETIMEOUT, "a bounded device-side wait gave up");
  }
  return NMFA_OK;
}

// The allocation-free variant of nmfa_run_device for the tensor path: the kernel's
// scratch comes from a static device array (see launch_tc_static_scratch) and signs
// must be supplied by the caller, so this path allocates no device memory.  (The
// launch plan is still built in host vectors.)
int nmfa_run_device_noalloc(nmfa_problem* p, const double* T_dev, int32_t t_f, double sigma, double alpha,
                            int32_t replicas, uint64_t seed, uint32_t stream_id, int8_t* signs_dev,
                            double* energy_dev, int64_t* energy_i64_dev, void* cuda_stream) {
  if (p == nullptr) return set_error(NMFA_EINVAL, "NULL handle");
  if (p->precision != NMFA_BF16 && p->precision != NMFA_BF16_FP8J)
    return set_error(NMFA_EUNSUPPORTED, "nmfa_run_device_noalloc takes NMFA_BF16 or NMFA_BF16_FP8J problems");
  if (signs_dev == nullptr) return set_error(NMFA_EINVAL, "nmfa_run_device_noalloc needs a signs buffer");
  if (t_f < 0 || (t_f > 0 && T_dev == nullptr)) return set_error(NMFA_EINVAL, "bad t_f or T");
  if (!(sigma >= 0.0) || !std::isfinite(sigma)) return set_error(NMFA_EINVAL, "sigma must be >= 0");
  if (!(alpha > 0.0 && alpha <= 1.0)) return set_error(NMFA_EINVAL, "alpha must be in (0, 1]");
  if (replicas < 1) return set_error(NMFA_EINVAL, "replicas must be >= 1");
  if (energy_i64_dev != nullptr && !p->integer_valued)
    return set_error(NMFA_EINVAL, "integer energies requested for a real-valued problem");
  std::lock_guard<std::mutex> g(p->mu);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int rc;
  if ((rc = cuda_error(cudaSetDevice(p->device), "cudaSetDevice"))) return rc;
  // Inside a stream capture the call becomes part of the caller's graph, which orders
  // it: the handle's completion event (recorded outside the capture) is neither waited
  // for nor recorded then.
  cudaStreamCaptureStatus capturing = cudaStreamCaptureStatusNone;
  if ((rc = cuda_error(cudaStreamIsCapturing(st, &capturing), "capture query"))) return rc;
  const bool in_capture = capturing != cudaStreamCaptureStatusNone;
  if (!in_capture && (rc = cuda_error(cudaStreamWaitEvent(st, p->done, 0), "stream wait"))) return rc;
  RunParams rp{};
  rp.T = T_dev;
  rp.t_f = t_f;
  rp.sigma = sigma;
  rp.alpha = alpha;
  rp.replicas = replicas;
  rp.seed = seed;
  rp.stream_id = stream_id;
  rp.noise_sign = 1;
  rp.signs = signs_dev;
  rp.energy = energy_dev;
  rp.energy_i64 = energy_i64_dev;
  TcProblem pb{};
  pb.n = p->n;
  pb.n_pad = p->n_pad;
  pb.Jq = p->Jq;
  pb.fp8 = p->precision == NMFA_BF16_FP8J;  // read as stored, widened in the kernel: no scratch for J
  pb.inv_d32 = p->inv_d32;
  pb.h32 = p->h32;
  pb.energy_exact = p->energy_exact;
  if ((rc = launch_tc_static_scratch(pb, rp, p->status, st))) return rc;
  if (!tc_fuses_energy(pb, rp) && (energy_dev != nullptr || energy_i64_dev != nullptr)) {
    EnergyProblem ep{};
    ep.n = p->n;
    ep.J8 = p->J8;
    ep.J64 = p->J64;
    ep.h = p->h64;
    ep.integer_valued = p->integer_valued;
    if ((rc = launch_energy(ep, signs_dev, replicas, energy_dev, energy_i64_dev, st))) return rc;
  }
  return in_capture ? NMFA_OK : cuda_error(cudaEventRecord(p->done, st), "event record");
}

// ---------------------------------------------------------------------------
// Batches: many tensor-path runs (different instances, sizes, replica counts,
// schedules) in one persistent launch.
// ---------------------------------------------------------------------------
struct nmfa_batch {
  std::vector<nmfa_problem*> problems;
  std::vector<nmfa_job> jobs;
  std::vector<int> bn;
  std::vector<DevBuf> ws;   // one workspace per plan
  std::vector<DevBuf> widened;  // BF16 copies of FP8-stored problems widened once (one per problem)
  DevBuf signs;             // sign scratch for jobs that did not supply a buffer
  std::vector<int8_t*> signs_ptr;
  std::vector<char> energy_fused;  // per job: energies formed inside the persistent kernel
  int32_t* status = nullptr;
  std::vector<TcPlan> plans;  // one persistent launch per tile width in the batch
  std::vector<std::vector<int32_t>> plan_jobs;  // per plan: the batch index of each of its jobs
  cudaStream_t own = nullptr;
  cudaEvent_t done = nullptr;
  // plans 1.. run beside plan 0 on their own streams when all their CTAs fit the
  // GPU together (fork / join events); otherwise one after the other
  bool concurrent = false;
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> side_done;
  cudaEvent_t fork = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int device = 0;
  std::mutex mu;
};

static void free_batch(nmfa_batch* b) {
  if (b == nullptr) return;
  if (b->done) cudaEventSynchronize(b->done);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (DevBuf& w : b->ws) pool_free(w.p);
  for (DevBuf& w : b->widened) pool_free(w.p);
  pool_free(b->signs.p);
  pool_free(b->status);
  if (b->done) cudaEventDestroy(b->done);
  if (b->fork) cudaEventDestroy(b->fork);
  for (cudaEvent_t e : b->side_done) cudaEventDestroy(e);
  for (cudaStream_t x : b->side) cudaStreamDestroy(x);
  if (b->own) cudaStreamDestroy(b->own);
  delete b;
}

// Enqueues the batch's work (flag reset, the persistent kernel, one energy kernel
// per job) on `st`; the plan was uploaded at creation.
static int batch_enqueue(nmfa_batch* b, cudaStream_t st) {
  int rc;
  if (b->concurrent) {
    // fork: plans 1.. on the side streams after everything before on `st`; join
    // before the energy kernels
    if ((rc = cuda_error(cudaEventRecord(b->fork, st), "fork"))) return rc;
    for (size_t k = 1; k < b->plans.size(); ++k) {
      cudaStream_t x = b->side[k - 1];
      if ((rc = cuda_error(cudaStreamWaitEvent(x, b->fork, 0), "fork wait"))) return rc;
      if ((rc = tc_enqueue_plan(b->plans[k], false, x))) return rc;
      if ((rc = cuda_error(cudaEventRecord(b->side_done[k - 1], x), "join"))) return rc;
    }
    if ((rc = tc_enqueue_plan(b->plans[0], false, st))) return rc;
    for (size_t k = 1; k < b->plans.size(); ++k)
      if ((rc = cuda_error(cudaStreamWaitEvent(st, b->side_done[k - 1], 0), "join wait"))) return rc;
  } else {
    for (const TcPlan& plan : b->plans)
      if ((rc = tc_enqueue_plan(plan, false, st))) return rc;
  }
  for (size_t j = 0; j < b->jobs.size(); ++j) {
    const nmfa_job& jb = b->jobs[j];
    if (b->energy_fused[j] || (jb.energy_dev == nullptr && jb.energy_i64_dev == nullptr)) continue;
    nmfa_problem* p = b->problems[j];
    EnergyProblem ep{};
    ep.n = p->n;
    ep.J8 = p->J8;
    ep.J64 = p->J64;
    ep.h = p->h64;
    ep.integer_valued = p->integer_valued;
    if ((rc = launch_energy(ep, b->signs_ptr[j], jb.replicas, jb.energy_dev, jb.energy_i64_dev, st))) return rc;
  }
  return NMFA_OK;
}

int nmfa_batch_create(nmfa_problem* const* problems, const nmfa_job* jobs, int32_t count, int32_t options,
                      nmfa_batch** out) {
  if (out == nullptr) return set_error(NMFA_EINVAL, "out is NULL");
  *out = nullptr;
  if (count < 1 || problems == nullptr || jobs == nullptr) return set_error(NMFA_EINVAL, "empty batch");
  for (int32_t j = 0; j < count; ++j) {
    const nmfa_problem* p = problems[j];
    const nmfa_job& jb = jobs[j];
    if (p == nullptr) return set_error(NMFA_EINVAL, "NULL problem in batch");
    if (p->precision != NMFA_BF16 && p->precision != NMFA_BF16_FP8J)
      return set_error(NMFA_EUNSUPPORTED, "batches take NMFA_BF16 or NMFA_BF16_FP8J problems");
    if (jb.t_f < 0 || (jb.t_f > 0 && jb.T_dev == nullptr)) return set_error(NMFA_EINVAL, "bad t_f or T in batch");
    if (!(jb.sigma >= 0.0) || !(jb.alpha > 0.0 && jb.alpha <= 1.0) || jb.replicas < 1)
      return set_error(NMFA_EINVAL, "bad sigma, alpha or replicas in batch");
    if (jb.energy_i64_dev != nullptr && !p->integer_valued)
      return set_error(NMFA_EINVAL, "integer energies requested for a real-valued problem");
    if (p->device != problems[0]->device) return set_error(NMFA_EINVAL, "batch problems live on different devices");
  }
  nmfa_batch* b = new nmfa_batch();
  auto fail = [&](int code) {
    std::string msg = t_last_error;
    free_batch(b);
    t_last_error = msg;
    return code;
  };
  b->problems.assign(problems, problems + count);
  b->jobs.assign(jobs, jobs + count);
  b->device = problems[0]->device;
  int rc;
  if ((rc = cuda_error(cudaSetDevice(b->device), "cudaSetDevice"))) return fail(rc);
  if ((rc = cuda_error(cudaStreamCreateWithFlags(&b->own, cudaStreamNonBlocking), "stream"))) return fail(rc);
  if ((rc = cuda_error(cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming), "event"))) return fail(rc);
  if ((rc = pool_alloc(reinterpret_cast<void**>(&b->status), 4))) return fail(rc);
  if ((rc = cuda_error(cudaMemset(b->status, 0, 4), "status"))) return fail(rc);
  size_t sign_bytes = 0;
  for (int32_t j = 0; j < count; ++j)
    if (jobs[j].signs_dev == nullptr) sign_bytes += static_cast<size_t>(jobs[j].replicas) * problems[j]->n;
  if (sign_bytes && (rc = ensure_buf(b->signs, sign_bytes))) return fail(rc);
  std::vector<TcJob> tj(count);
  size_t sp = 0;
  b->signs_ptr.resize(count);
  std::vector<const nmfa_problem*> widened_of;  // the problem each widened copy belongs to
  for (int32_t j = 0; j < count; ++j) {
    nmfa_problem* p = problems[j];
    const nmfa_job& jb = jobs[j];
    int8_t* sg = jb.signs_dev;
    if (sg == nullptr) {
      sg = static_cast<int8_t*>(b->signs.p) + sp;
      sp += static_cast<size_t>(jb.replicas) * p->n;
    }
    b->signs_ptr[j] = sg;
    TcJob& t = tj[j];
    t.pb.n = p->n;
    t.pb.n_pad = p->n_pad;
    t.pb.Jq = p->Jq;
    t.pb.fp8 = p->precision == NMFA_BF16_FP8J;  // read as stored (E4M3), widened to BF16 in the kernel
    if (t.pb.fp8 && p->n_pad <= kFp8WidenOnceMaxNpad && !(options & NMFA_BATCH_FP8_IN_KERNEL)) {
      // small and mid-size FP8 problems: one BF16 copy per problem for the batch's
      // lifetime, and the BF16 kernel (bit-identical runs)
      size_t w = 0;
      while (w < widened_of.size() && widened_of[w] != p) ++w;
      if (w == widened_of.size()) {
        b->widened.emplace_back();
        if ((rc = ensure_buf(b->widened.back(), 2 * static_cast<size_t>(p->n_pad) * p->n_pad))) return fail(rc);
        if ((rc = launch_widen_e4m3(p->Jq, b->widened.back().p, p->n_pad, b->own))) return fail(rc);
        widened_of.push_back(p);
      }
      t.pb.Jq = b->widened[w].p;
      t.pb.fp8 = false;
    }
    t.pb.inv_d32 = p->inv_d32;
    t.pb.h32 = p->h32;
    t.pb.energy_exact = p->energy_exact;
    t.rp = RunParams{};
    t.rp.T = jb.T_dev;
    t.rp.t_f = jb.t_f;
    t.rp.sigma = jb.sigma;
    t.rp.alpha = jb.alpha;
    t.rp.replicas = jb.replicas;
    t.rp.seed = jb.seed;
    t.rp.stream_id = jb.stream_id;
    t.rp.noise_sign = 1;
    t.rp.signs = sg;
    t.rp.energy = jb.energy_dev;
    t.rp.energy_i64 = jb.energy_i64_dev;
    b->energy_fused.push_back(tc_fuses_energy(t.pb, t.rp) ? 1 : 0);
    t.bn = (options & NMFA_BATCH_BN64) ? 64
           : (options & (NMFA_BATCH_BN128 | NMFA_BATCH_PAIR128)) ? 128
           : (options & NMFA_BATCH_BN256) ? 256
           : ((options & NMFA_BATCH_AUTOTUNE) && p->precision == NMFA_BF16) ? nmfa_autotuned_bn(p, jb.replicas)
                                             : tc_pick_bn_for(t.pb, jb.replicas);
    // CTA pairs only on request (where the problem allows them; not with FP8 couplings)
    t.pair = (options & NMFA_BATCH_PAIR128) && !t.pb.fp8 && tc_use_pair(t.bn, p->n_pad);
    b->bn.push_back(t.bn);
  }
  // one persistent launch per tile variant present in the batch
  struct Variant {
    int bn;
    bool pair, f8;
  };
  const Variant variants[] = {{256, false, false}, {256, false, true}, {128, true, false},
                              {128, false, false}, {128, false, true}, {64, false, false}, {64, false, true}};
  for (const Variant& var : variants) {
    std::vector<TcJob> part;
    std::vector<int32_t> part_jobs;
    for (size_t j = 0; j < tj.size(); ++j) {
      const TcJob& t = tj[j];
      if (t.bn == var.bn && t.pair == var.pair && t.pb.fp8 == var.f8) {
        part.push_back(t);
        part_jobs.push_back(static_cast<int32_t>(j));
      }
    }
    if (part.empty()) continue;
    int64_t bytes = 0;
    if ((rc = tc_plan_bytes(part.data(), static_cast<int32_t>(part.size()), &bytes))) return fail(rc);
    b->ws.emplace_back();
    if ((rc = ensure_buf(b->ws.back(), static_cast<size_t>(bytes)))) return fail(rc);
    b->plans.emplace_back();
    b->plan_jobs.push_back(part_jobs);
    const bool withhold = (options & NMFA_BATCH_DEBUG_WITHHOLD_TILE) && b->plans.size() == 1;  // the first plan
    if (withhold && part[0].pb.n_pad <= 128) return fail(set_error(NMFA_EINVAL, "withheld tile needs n > 128"));
    if ((rc = tc_build_plan(part.data(), static_cast<int32_t>(part.size()), b->ws.back().p, bytes, b->status,
                            &b->plans.back(), withhold)))
      return fail(rc);
    // upload the plan once (kernel-parameter copies on the batch's stream)
    if ((rc = tc_upload_plan(b->plans.back(), b->own))) return fail(rc);
  }
  if ((rc = cuda_error(cudaStreamSynchronize(b->own), "plan upload"))) return fail(rc);
  if (b->plans.size() > 1) {
    // Concurrent plans need all their CTAs resident at once (each CTA holds an SM's
    // tensor memory): otherwise a later plan's groups could start partly and wait
    // for the rest of their tiles until an earlier plan ends.
    int sms = 0, total = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    for (const TcPlan& pl : b->plans) total += pl.grid;
    if (sms > 0 && total <= sms) {
      b->concurrent = true;
      if ((rc = cuda_error(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming), "event"))) return fail(rc);
      for (size_t k = 1; k < b->plans.size(); ++k) {
        b->side.emplace_back();
        if ((rc = cuda_error(cudaStreamCreateWithFlags(&b->side.back(), cudaStreamNonBlocking), "stream")))
          return fail(rc);
        b->side_done.emplace_back();
        if ((rc = cuda_error(cudaEventCreateWithFlags(&b->side_done.back(), cudaEventDisableTiming), "event")))
          return fail(rc);
      }
    }
  }
  if (options & NMFA_BATCH_GRAPH) {
    if ((rc = cuda_error(cudaStreamBeginCapture(b->own, cudaStreamCaptureModeThreadLocal), "capture"))) return fail(rc);
    rc = batch_enqueue(b, b->own);
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamEndCapture(b->own, &g);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return fail(rc);
    }
    if ((rc = cuda_error(ce, "end capture"))) return fail(rc);
    b->graph = g;
    if ((rc = cuda_error(cudaGraphInstantiate(&b->exec, g, 0), "graph instantiate"))) return fail(rc);
  }
  *out = b;
  return NMFA_OK;
}

int nmfa_batch_launch(nmfa_batch* b, void* cuda_stream) {
  if (b == nullptr) return set_error(NMFA_EINVAL, "NULL batch");
  std::lock_guard<std::mutex> g(b->mu);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int rc;
  if ((rc = cuda_error(cudaSetDevice(b->device), "cudaSetDevice"))) return rc;
  if ((rc = cuda_error(cudaStreamWaitEvent(st, b->done, 0), "stream wait"))) return rc;
  if (b->exec != nullptr) {
    if ((rc = cuda_error(cudaGraphLaunch(b->exec, st), "graph launch"))) return rc;
    count_launch(1);
  } else if ((rc = batch_enqueue(b, st))) {
    return rc;
  }
  return cuda_error(cudaEventRecord(b->done, st), "event record");
}

int nmfa_batch_set_stream_ids(nmfa_batch* b, const uint32_t* stream_ids, int32_t count) {
  if (b == nullptr || stream_ids == nullptr) return set_error(NMFA_EINVAL, "NULL argument");
  if (count != static_cast<int32_t>(b->jobs.size())) return set_error(NMFA_EINVAL, "one stream id per job");
  std::lock_guard<std::mutex> g(b->mu);
  int rc;
  if ((rc = cuda_error(cudaSetDevice(b->device), "cudaSetDevice"))) return rc;
  // the new descriptors replace the old ones after the last launch has finished
  if ((rc = cuda_error(cudaStreamWaitEvent(b->own, b->done, 0), "stream wait"))) return rc;
  for (size_t k = 0; k < b->plans.size(); ++k) {
    std::vector<uint32_t> ids;
    for (int32_t j : b->plan_jobs[k]) ids.push_back(stream_ids[j]);
    tc_plan_set_streams(&b->plans[k], ids.data());
    if ((rc = tc_upload_plan(b->plans[k], b->own))) return rc;
  }
  for (int32_t j = 0; j < count; ++j) b->jobs[j].stream_id = stream_ids[j];
  return cuda_error(cudaEventRecord(b->done, b->own), "event record");
}

int nmfa_batch_sync(nmfa_batch* b) {
  if (b == nullptr) return set_error(NMFA_EINVAL, "NULL batch");
  int rc = cuda_error(cudaEventSynchronize(b->done), "sync");
  if (rc) return rc;
  int32_t st = 0;
  if ((rc = cuda_error(cudaMemcpy(&st, b->status, 4, cudaMemcpyDeviceToHost), "status read"))) return rc;
  if (st != kStatusOk) {
    cudaMemset(b->status, 0, 4);
    return set_error(NMFA_ETIMEOUT, "a bounded device-side wait gave up");
  }
  return NMFA_OK;
}

int nmfa_batch_info(const nmfa_batch* b, int32_t* grid, int32_t* groups, int64_t* workspace_bytes) {
  if (b == nullptr) return set_error(NMFA_EINVAL, "NULL batch");
  if (grid) {
    int32_t gmax = 0;
    for (const TcPlan& pl : b->plans) gmax = std::max<int32_t>(gmax, pl.grid);
    *grid = gmax;
  }
  if (groups) {
    int32_t g = 0;
    for (size_t j = 0; j < b->jobs.size(); ++j) g += (b->jobs[j].replicas + b->bn[j] - 1) / b->bn[j];
    *groups = g;
  }
  if (workspace_bytes) {
    size_t tot = b->signs.bytes;
    for (const DevBuf& w : b->ws) tot += w.bytes;
    for (const DevBuf& w : b->widened) tot += w.bytes;
    *workspace_bytes = static_cast<int64_t>(tot);
  }
  return NMFA_OK;
}

void nmfa_batch_destroy(nmfa_batch* b) { free_batch(b); }

int nmfa_batch_plan(const nmfa_batch* b, int32_t* bn, int32_t* ctas_per_mma, int32_t* cluster_ctas, int32_t capacity,
                    int32_t* count) {
  if (b == nullptr) return set_error(NMFA_EINVAL, "NULL batch");
  const int32_t n = static_cast<int32_t>(b->plans.size());
  for (int32_t k = 0; k < n && k < capacity; ++k) {
    if (bn) bn[k] = b->plans[k].bn;
    if (ctas_per_mma) ctas_per_mma[k] = b->plans[k].pair ? 2 : 1;
    if (cluster_ctas) cluster_ctas[k] = b->plans[k].pair ? 2 : 1;
  }
  if (count) *count = n;
  return NMFA_OK;
}

// Tuning hook for the CUDA-core paths (replicas per CTA: 0 = automatic, else 1/2/4/8).
int nmfa_debug_withhold_arrival(nmfa_problem* p, int32_t step) {
  if (p == nullptr) return set_error(NMFA_EINVAL, "NULL handle");
  if (step < -1) return set_error(NMFA_EINVAL, "step must be >= -1");
  p->withhold_step = step;
  return NMFA_OK;
}

int nmfa_tune_replicas_per_cta(nmfa_problem* p, int32_t rc) {
  if (p == nullptr) return set_error(NMFA_EINVAL, "NULL handle");
  if (rc != 0 && rc != 1 && rc != 2 && rc != 4 && rc != 8) return set_error(NMFA_EINVAL, "rc must be 0, 1, 2, 4 or 8");
  p->replicas_per_cta = rc;
  return NMFA_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Autotuner: replicas per tile (bn = 64, 128 or 256) for the tensor path, chosen by
// timing a short run of each candidate on the problem itself and cached by the
// run's shape (n_pad, replicas) only, so that an instance's tiling (and hence
// its results) never depends on what else shares a batch.  Results are identical
// for either choice; the tuner only trades tile count against tile width.
// ---------------------------------------------------------------------------
#include <map>
static std::mutex g_tune_mu;
static std::map<std::pair<int, int>, int> g_tune_cache;

static int nmfa_autotuned_bn(nmfa_problem* p, int32_t replicas) {
  if (replicas <= 64 || p->precision != NMFA_BF16) return tc_pick_bn(replicas, p->n_pad);
  const std::pair<int, int> key(p->n_pad, replicas);
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) return it->second;
  }
  int best = tc_pick_bn(replicas, p->n_pad);
  float best_ms = 1e30f;
  const int t_f = 24;
  double* T = nullptr;
  int8_t* signs = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  DevBuf ws;
  bool okc = pool_alloc(reinterpret_cast<void**>(&T), sizeof(double) * t_f) == NMFA_OK &&
             pool_alloc(reinterpret_cast<void**>(&signs), static_cast<size_t>(replicas) * p->n) == NMFA_OK &&
             cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
  if (okc) {
    std::vector<double> Th(t_f, 1.0);
    okc = cudaMemcpy(T, Th.data(), sizeof(double) * t_f, cudaMemcpyHostToDevice) == cudaSuccess;
  }
  for (int bn : {64, 128, 256}) {
    if (bn == 256 && replicas <= 128) continue;
    if (!okc) break;
    TcJob jb{};
    jb.pb.n = p->n;
    jb.pb.n_pad = p->n_pad;
    jb.pb.Jq = p->Jq;
    jb.pb.inv_d32 = p->inv_d32;
    jb.pb.h32 = p->h32;
    jb.rp.T = T;
    jb.rp.t_f = t_f;
    jb.rp.sigma = 0.15;
    jb.rp.alpha = 0.15;
    jb.rp.replicas = replicas;
    jb.rp.noise_sign = 1;
    jb.rp.signs = signs;
    jb.bn = bn;
    int64_t bytes = 0;
    TcPlan plan;
    if (tc_plan_bytes(&jb, 1, &bytes) || ensure_buf(ws, static_cast<size_t>(bytes)) ||
        tc_build_plan(&jb, 1, ws.p, bytes, p->status, &plan))
      continue;
    float ms = 0.0f;
    bool good = tc_enqueue_plan(plan, true, st) == NMFA_OK && cudaStreamSynchronize(st) == cudaSuccess;
    for (int rep = 0; rep < 2 && good; ++rep) {
      good = cudaEventRecord(e0, st) == cudaSuccess && tc_enqueue_plan(plan, true, st) == NMFA_OK &&
             cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
             cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
    }
    if (good && ms < best_ms) {
      best_ms = ms;
      best = bn;
    }
  }
  pool_free(ws.p);
  pool_free(T);
  pool_free(signs);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  cudaGetLastError();
  std::lock_guard<std::mutex> g(g_tune_mu);
  g_tune_cache[key] = best;
  return best;
}

extern "C" int nmfa_autotune_bn(nmfa_problem* p, int32_t replicas, int32_t* bn) {
  if (p == nullptr || bn == nullptr || replicas < 1) return set_error(NMFA_EINVAL, "bad autotune arguments");
  if (p->precision != NMFA_BF16) return set_error(NMFA_EUNSUPPORTED, "autotuning is for NMFA_BF16 problems");
  std::lock_guard<std::mutex> g(p->mu);
  *bn = nmfa_autotuned_bn(p, replicas);
  return NMFA_OK;
}
