// nmfa_internal.h -- structures shared between the C-ABI layer and the kernels.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include "nmfa.h"

namespace nmfa {

// Process-wide count of kernel launches made by the library.
extern std::atomic<uint64_t> g_launches;
inline void count_launch(uint64_t k = 1) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// Thread-local error message; returns `code` for convenience.
int set_error(int code, const std::string& msg);
int cuda_error(cudaError_t e, const char* where);

// Device memory of the library comes from the current device's stream-ordered pool,
// which keeps freed memory for reuse: neither call synchronises the device (cudaFree
// waits for all work on the device, which stalled a serving loop's launches behind
// its releases).  pool_alloc returns memory usable on any stream.  pool_free releases
// `p` once `after` (an event recorded after the buffer's last use, or nullptr when
// the host has already seen that use complete) has completed.
int pool_alloc(void** p, size_t bytes);
void pool_free(void* p, cudaEvent_t after = nullptr);

// Device-side status word written by kernels with bounded waits.
enum DeviceStatus : int32_t { kStatusOk = 0, kStatusTimeout = 1 };

// One run's parameters as the kernels see them.
struct RunParams {
  const double* T;        // device, t_f temperatures
  int32_t t_f;
  double sigma;
  double alpha;
  int32_t replicas;
  uint64_t seed;
  uint32_t stream_id;
  int32_t noise_sign;
  const double* s0;       // device R*n or nullptr
  double* s_out;          // device R*n or nullptr
  double* phi_out;        // device R*n or nullptr
  int8_t* signs;          // device R*n (always present: the library supplies scratch)
  // Energies of the sign vectors (Eq. 1), device R, or nullptr.  The tensor path
  // computes them inside its persistent kernel when the problem allows it exactly
  // (TcProblem::energy_exact); every other path leaves them to launch_energy.
  double* energy;
  int64_t* energy_i64;
};

// ---- CUDA-core dense path (FP32 / FP64) -----------------------------------
struct DenseSimtProblem {
  int32_t n;
  int32_t ldj;            // row stride of J in elements (n for FP64; n rounded up to 128 for FP32)
  const void* J;          // float or double, row-major, symmetric; FP32 J is n_pad x n_pad, zero-padded
  const void* h;          // float or double, n (zeros when h = 0)
  const double* d;        // FP64 row norms
  const float* inv_d32;   // 1/d_i in binary32 (0 where d_i = 0)
};
int launch_dense_simt(bool fp64, const DenseSimtProblem& pb, const RunParams& rp,
                      cudaStream_t st, int replicas_per_cta);
// FP32 dense path for large n: the whole run in one cooperative launch (register-
// blocked GEMM tiles, split along K when the tiles are fewer than the CTAs, fused
// update, a grid barrier per step).  State, partial tiles and counters live in a
// caller-provided scratch of tiled_f32_workspace_bytes(n, R) bytes; bounded waits
// report through `status`.  withhold_step >= 0: the first CTA does not arrive at the
// grid barrier closing that step (a test of the bounded waits).
int64_t tiled_f32_workspace_bytes(int32_t n, int32_t replicas);
int launch_dense_tiled_f32(const DenseSimtProblem& pb, const RunParams& rp, void* ws, int32_t* status,
                           int32_t withhold_step, cudaStream_t st);
// Which FP32 dense problems take the tiled kernel: from n = 256 spins, and above
// n = 128 when there are more than 512 replicas.  Below that the replica-resident
// kernel (no grid barrier) is faster; above it that kernel's per-spin loop over n
// couplings read from L2 sets the step time (measured on GB300, 1000-step runs, ms,
// replica-resident against tiled for R = 64 / 256 / 1024: n = 128: 1.6 / 1.9 / 2.6
// against 7.7 / 8.3 / 8.3; n = 192: 3.2 / 4.1 / 15.2 against 7.3 / 7.5 / 10.4;
// n = 256: 19.9 / 20.8 / 21.6 against 7.5 / 7.4 / 10.5; n = 384: 60.6 / 61.1 / 63.3
// against 7.7 / 7.8 / 15.2).
inline bool tiled_f32_preferred(int32_t n, int32_t replicas) { return n >= 256 || (n > 128 && replicas > 512); }

// ---- CUDA-core CSR path (FP32 / FP64) ---------------------------------------
struct CsrProblem {
  int32_t n;
  int32_t nnz;
  const int32_t* row_ptr; // n+1
  const int32_t* col;     // nnz
  const void* val;        // float/double nnz, or int8 when val_int8
  bool val_int8;
  const void* h;
  const double* d;
  const float* inv_d32;
};
int launch_csr(bool fp64, const CsrProblem& pb, const RunParams& rp, cudaStream_t st,
               int replicas_per_cta);

// Arithmetic throughput of the current device, timed with CUDA events on `st`
// (synchronous): kind 0 = FP32 FMA, 1 = FP64 FMA (TFLOP/s, 2 flops per FMA),
// 2 = tanh.approx.f32 on the MUFU (Tops/s).
int measure_alu_peak(int kind, cudaStream_t st, double* rate);

// ---- Eq. (1) energies from signs --------------------------------------------
struct EnergyProblem {
  int32_t n;
  const int8_t* J8;       // int8 copy (integer problems with |J| <= 127) or nullptr
  const double* J64;      // FP64 copy (used when J8 is null)
  const int32_t* row_ptr; // CSR form (used when non-null)
  const int32_t* col;
  const double* val64;
  const double* h;        // FP64 fields or nullptr
  bool integer_valued;
};
int launch_energy(const EnergyProblem& ep, const int8_t* signs, int32_t replicas,
                  double* energy, int64_t* energy_i64, cudaStream_t st);

// ---- preparation kernels ------------------------------------------------------
int launch_row_norms_dense(int32_t n, const double* J64, const double* h, double* d,
                           float* inv_d32, cudaStream_t st);
int launch_row_norms_csr(int32_t n, const int32_t* row_ptr, const double* val64,
                         const double* h, double* d, float* inv_d32, cudaStream_t st);
// dst[i*ld + j] = convert(J64[i*n + j]) for i,j < n, zero in the padding up to
// rows x ld.  kind: 0 = float, 1 = bf16, 2 = e4m3, 3 = int8.
int launch_convert_dense(int32_t n, const double* J64, void* dst, int kind, int64_t rows,
                         int64_t ld, cudaStream_t st);
// BF16 n_pad x n_pad couplings (natural order) from their E4M3 storage (each group of
// four values stored as k0, k2, k1, k3); exact.
int launch_widen_e4m3(const void* Jq8, void* Jq16, int64_t n_pad, cudaStream_t st);
// FP8-stored problems up to this n_pad are widened to BF16 once per batch (a scratch
// copy of 2 n_pad^2 bytes) instead of slice by slice in the kernel every step: the
// kernel's converter warps cost 1.2-1.6x the step time there (measured on GB300,
// SK, 200 steps: n = 1024, R = 512 1.19x; n = 2000, R = 1024 1.45x; n = 4096, R = 512
// 1.58x), while the copy is at most 32 MB.  Larger problems are read as stored.
constexpr int32_t kFp8WidenOnceMaxNpad = 4096;
int launch_convert_vec(int32_t n, const double* src, void* dst, int kind, cudaStream_t st);

// ---- tcgen05 tensor path ------------------------------------------------------
struct TcProblem {
  int32_t n;
  int32_t n_pad;          // spins padded to a multiple of 128 (rows and K)
  const void* Jq;         // BF16 [n_pad][n_pad] or (fp8) E4M3 [n_pad][n_pad], read by the kernel as stored
  bool fp8;
  const float* inv_d32;   // n_pad, 0 in padding
  const float* h32;       // h_i in binary32, n_pad (0 in padding)
  // Integer J and h with max_i (sum_j |J_ij| + 2 |h_i|) < 2^24: the product J s~ + 2h
  // of a sign vector is exact in the FP32 accumulator, so the kernel can form the
  // energies itself.
  bool energy_exact;
};
// True when the tensor kernel forms this run's energies (no separate energy launch).
inline bool tc_fuses_energy(const TcProblem& pb, const RunParams& rp) {
  return pb.energy_exact && rp.t_f > 0 && (rp.energy != nullptr || rp.energy_i64 != nullptr);
}
struct TcWorkspace {
  void* S16;              // bf16 [2][r_pad][n_pad]
  uint32_t* flags;        // [row blocks][replica blocks]
  int32_t* status;
  int64_t bytes;
};
int tc_workspace_bytes(const TcProblem& pb, int32_t replicas, int64_t* bytes);
// One instance run on the tensor path, and a launch plan for a batch of them.
struct TcJob {
  TcProblem pb;
  RunParams rp;
  int bn;                  // replicas per tile: 64, 128 or 256
  bool pair = false;       // 128-replica tiles as CTA pairs (cta_group::2 MMAs of M = 256)
};
struct TcPlan {
  std::vector<unsigned char> host;   // group descriptors, items, per-CTA offsets
  std::vector<int32_t> group_job;    // index (into the plan's jobs) of each group's job
  void* dev = nullptr;               // workspace base
  size_t groups_off = 0, items_off = 0, first_off = 0, flags_off = 0, flags_bytes = 0;
  int grid = 0;                      // CTAs launched
  int bn = 128;
  bool pair = false;
  bool f8 = false;
  int32_t* status = nullptr;
  double makespan = 0.0;             // scheduler's estimate (relative units)
};
// Default replicas per tile (64, 128 or 256) of a run of `replicas` replicas of an n_pad problem.
int tc_pick_bn(int32_t replicas, int32_t n_pad);
// The same for this problem's storage (FP8-stored couplings take the same widths).
int tc_pick_bn_for(const TcProblem& pb, int32_t replicas);
// Whether 128-replica tiles of an n_pad problem run as CTA pairs (results do not change).
bool tc_use_pair(int bn, int32_t n_pad);
int tc_plan_bytes(const TcJob* jobs, int32_t count, int64_t* bytes);
// withhold_tile (test only): leave group 0's last row-block tile out of the work lists.
int tc_build_plan(const TcJob* jobs, int32_t count, void* ws, int64_t ws_bytes, int32_t* status, TcPlan* plan,
                  bool withhold_tile = false);
int tc_upload_plan(const TcPlan& plan, cudaStream_t st);
// Sets the noise stream id of every group of the plan's job j to stream_ids[j] (host
// copy of the descriptors; upload it before the next launch).
void tc_plan_set_streams(TcPlan* plan, const uint32_t* stream_ids);
int tc_enqueue_plan(const TcPlan& plan, bool upload, cudaStream_t st);
int launch_tc(const TcProblem& pb, const RunParams& rp, const TcWorkspace& ws,
              cudaStream_t st);
// Same launch with the scratch taken from a fixed-size static device array.
int launch_tc_static_scratch(const TcProblem& pb, const RunParams& rp, int32_t* status,
                             cudaStream_t st);

}  // namespace nmfa
