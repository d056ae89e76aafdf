// k_tc.cu -- the tcgen05 tensor-core path of NMFA (BF16 J and S, FP32 accumulation).
//
// One persistent launch runs all t_f steps of Algorithm 1 for a batch of replicas.
// The coupling product of line 6 over all replicas is the GEMM P = J S (J: n x n,
// S: n x R); CTA (b, c) owns the output tile of spins [128 b, 128 b + 128) and
// replicas [BN c, BN c + BN) for the whole run:
//   - warp 0 streams 64-wide K slices of J's row block and of S's replica block
//     into a STAGES-deep shared-memory ring with TMA (128-byte swizzle); the J
//     slices of a step start before the step's state is published, the S slices
//     after the whole warp has seen every row block's epoch flag of the replica
//     block reach the step;
//   - warp 1 (one lane) issues tcgen05.mma (M = 128, N = BN, K = 16) into a TMEM
//     accumulator, releasing ring slots and the accumulator with tcgen05.commit;
//   - warps 2..17 first draw the step's noise (Philox/Box-Muller, independent of
//     the state) while the tensor core works and park sigma*z in TMEM; once the
//     accumulator is complete they read it with tcgen05.ld and finish the step:
//     normalisation by d_i, -tanh(Phi/T_t) and the alpha-mix into the FP32 master
//     state, which stays in TMEM for the whole run (line 10); the new state is
//     written in BF16 to the next of two global S buffers (L2-resident) and
//     published by bumping the tile's epoch flag.
// Step t+1's slices of row block b' are loaded only after tile (b', c) has
// published step t, which realises the synchronous update of Algorithm 1
// (every Phi from the old state) without a grid-wide barrier: only the CTAs of
// one replica block depend on one another.  After the last step the signs are
// read out from the FP32 master state (lines 13-15).
//
// Every wait (mbarrier or flag) is bounded by a 2-second wall-clock limit; on
// expiry the CTA records NMFA's timeout status, drains its own TMA copies and
// MMAs, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdio>
#include <mutex>

#include "nmfa_device.cuh"
#include "nmfa_internal.h"
#include "tc_ptx.cuh"

namespace nmfa {

namespace {

constexpr int kBM = 128;               // spins per tile (TMEM lanes)
constexpr int kBK = 64;                // K slice: 64 BF16 = one 128-byte swizzle row
constexpr int kEpiWarps = 16;          // four warps per TMEM lane quarter
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr uint64_t kTimeoutNs = 2000000000ull;
constexpr uint64_t kDrainNs = 200000000ull;

struct TcArgs {
  int32_t n, n_pad, r_pad, replicas, t_f, c_offset, rbk;
  const float* inv_d32;
  const float* h32;
  const double* T;
  float sigma_ns, alpha, one_m_alpha;
  NoiseKey key;
  uint32_t stream;
  const double* s0;
  double* s_out;
  double* phi_out;
  int8_t* signs;
  __nv_bfloat16* S16;   // [2][r_pad][n_pad]
  uint32_t* flags;      // [n_pad/128][rbk]
  int32_t* status;
};

struct SharedCtl {
  uint64_t full[16];
  uint64_t empty[16];
  uint64_t acc_full;
  uint64_t acc_empty;
  uint64_t drain;
  uint64_t epi_sync;   // rendezvous of the epilogue warps (bounded, abort-aware)
  uint32_t tmem_slot;
  int32_t abort_flag;
};

__device__ __forceinline__ void raise_abort(SharedCtl* ctl, int32_t* status) {
  *reinterpret_cast<volatile int32_t*>(&ctl->abort_flag) = 1;
  atomicExch(status, static_cast<int32_t>(kStatusTimeout));
}

__device__ __forceinline__ bool aborted(SharedCtl* ctl) {
  return *reinterpret_cast<volatile int32_t*>(&ctl->abort_flag) != 0;
}

// Bounded mbarrier wait; false if the run is being aborted.
__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity, SharedCtl* ctl, int32_t* status,
                                         uint64_t limit_ns = kTimeoutNs) {
  if (ptx::mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = ptx::globaltimer_ns();
  while (true) {
    if (ptx::mbar_try_wait(bar, parity)) return true;
    if (aborted(ctl)) return false;
    if (ptx::globaltimer_ns() - t0 > limit_ns) {
      raise_abort(ctl, status);
      return false;
    }
  }
}

// Warp-wide wait until every row block's epoch flag of one replica block reaches
// `need`: lane l polls row blocks l, l+32, ... in parallel (one round trip per poll
// instead of one per row block).  Returns false (on every lane) on abort/timeout.
__device__ __forceinline__ bool wait_group_flags(const uint32_t* f0, int nb, int stride, uint32_t need, int lane,
                                                 SharedCtl* ctl, int32_t* status) {
  const uint64_t t0 = ptx::globaltimer_ns();
  while (true) {
    bool mine = true;
    for (int rb = lane; rb < nb; rb += 32) mine = mine && (ptx::ld_acquire_gpu(f0 + static_cast<int64_t>(rb) * stride) >= need);
    if (__all_sync(0xffffffffu, mine)) return true;
    int stop = 0;
    if (lane == 0) {
      if (aborted(ctl)) {
        stop = 1;
      } else if (ptx::globaltimer_ns() - t0 > kTimeoutNs) {
        raise_abort(ctl, status);
        stop = 1;
      }
    }
    if (__shfl_sync(0xffffffffu, stop, 0)) return false;
  }
}

template <int BN>
struct TcCfg {
  static constexpr int kStages = BN >= 128 ? 6 : 8;
  static constexpr uint32_t kABytes = kBM * 128;
  static constexpr uint32_t kBBytes = BN * 128;
  static constexpr uint32_t kStageBytes = kABytes + kBBytes;
  // accumulator [0, BN), FP32 master state [BN, 2BN), the step's noise [2BN, 3BN)
  static constexpr uint32_t kTmemCols = (3 * BN <= 64 ? 64 : (3 * BN <= 128 ? 128 : (3 * BN <= 256 ? 256 : 512)));
  static constexpr size_t kSmemBytes = static_cast<size_t>(kStages) * kStageBytes + 1024;
  static_assert(kStages <= 16, "ring too deep");
  static_assert(BN % 32 == 0 && BN >= 64 && BN <= 256, "BN");
};

template <int BN>
__global__ void __launch_bounds__(kThreads, 1)
nmfa_tc_kernel(const __grid_constant__ CUtensorMap tmJ, const __grid_constant__ CUtensorMap tmS, TcArgs a) {
  using Cfg = TcCfg<BN>;
  constexpr int kStages = Cfg::kStages;
  extern __shared__ __align__(1024) uint8_t smem_dyn[];
  __shared__ SharedCtl ctl;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int b = blockIdx.x;
  const int c = a.c_offset + blockIdx.y;
  const int KB = a.n_pad / kBK;
  const uint32_t ring = (ptx::smem_u32(smem_dyn) + 1023u) & ~1023u;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      ptx::mbar_init(ptx::smem_u32(&ctl.full[s]), 1);
      ptx::mbar_init(ptx::smem_u32(&ctl.empty[s]), 1);
    }
    ptx::mbar_init(ptx::smem_u32(&ctl.acc_full), 1);
    ptx::mbar_init(ptx::smem_u32(&ctl.acc_empty), kEpiWarps);
    ptx::mbar_init(ptx::smem_u32(&ctl.drain), 1);
    ptx::mbar_init(ptx::smem_u32(&ctl.epi_sync), kEpiWarps);
    ctl.abort_flag = 0;
    ptx::fence_mbar_init();
    ptx::tma_prefetch_desc(&tmJ);
    ptx::tma_prefetch_desc(&tmS);
  }
  if (warp == 1) {
    ptx::tmem_alloc(ptx::smem_u32(&ctl.tmem_slot), Cfg::kTmemCols);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = ctl.tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    // Per step: claim the first ring slots and start their J slices at once (J
    // does not depend on the previous step), wait with the whole warp until every
    // row block of this replica block has published the step's state, then issue
    // the S slices of the claimed slots and stream the rest of the step.
    const int pre = KB < kStages ? KB : kStages;
    uint32_t it = 0;        // ring iterations whose J and S copies are both issued
    int pending = 0;        // claimed slots with only the J copy issued
    bool ok = true;
    auto kslice = [&](int kb) {
      int kbr = kb + 2 * b;
      return kbr >= KB ? kbr - KB : kbr;
    };
    for (int t = 0; t < a.t_f && ok; ++t) {
      const int buf = t & 1;
      const int sy = buf * a.r_pad + c * BN;
      if (lane == 0) {
        for (int kb = 0; kb < pre; ++kb) {
          const uint32_t k = it + kb, stage = k % kStages, phase = (k / kStages) & 1u;
          ok = wait_bar(ptx::smem_u32(&ctl.empty[stage]), phase ^ 1u, &ctl, a.status);
          if (!ok) break;
          const uint32_t full = ptx::smem_u32(&ctl.full[stage]);
          ptx::mbar_arrive_expect_tx(full, Cfg::kStageBytes);
          ptx::tma_load_2d(ring + stage * Cfg::kStageBytes, &tmJ, kslice(kb) * kBK, b * kBM, full);
          pending = kb + 1;
        }
      }
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      if (!ok) break;
      ok = wait_group_flags(a.flags + c, a.n_pad / kBM, a.rbk, static_cast<uint32_t>(t + 1), lane, &ctl, a.status);
      // each lane acquired its own row blocks' flags; the warp barrier orders those
      // acquires before lane 0's copies (memory ordering among the warp's threads)
      __syncwarp();
      if (lane == 0) {
        if (ok) ptx::fence_proxy_async_global();
        // the S halves of the claimed slots (also on abort, so that their barriers complete)
        for (int kb = 0; kb < pending; ++kb) {
          const uint32_t k = it + kb, stage = k % kStages;
          ptx::tma_load_2d(ring + stage * Cfg::kStageBytes + Cfg::kABytes, &tmS, kslice(kb) * kBK, sy,
                           ptx::smem_u32(&ctl.full[stage]));
        }
        it += pending;
        pending = 0;
        for (int kb = pre; kb < KB && ok; ++kb) {
          const uint32_t stage = it % kStages, phase = (it / kStages) & 1u;
          ok = wait_bar(ptx::smem_u32(&ctl.empty[stage]), phase ^ 1u, &ctl, a.status);
          if (!ok) break;
          const uint32_t full = ptx::smem_u32(&ctl.full[stage]);
          const uint32_t sA = ring + stage * Cfg::kStageBytes;
          ptx::mbar_arrive_expect_tx(full, Cfg::kStageBytes);
          ptx::tma_load_2d(sA, &tmJ, kslice(kb) * kBK, b * kBM, full);
          ptx::tma_load_2d(sA + Cfg::kABytes, &tmS, kslice(kb) * kBK, sy, full);
          ++it;
        }
      }
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
    }
    if (!ok && lane == 0) {
      // J-only slots claimed before a failed wait get their S copy so their barriers complete
      for (int kb = 0; kb < pending; ++kb) {
        const uint32_t k = it + kb, stage = k % kStages;
        ptx::tma_load_2d(ring + stage * Cfg::kStageBytes + Cfg::kABytes, &tmS, kslice(kb) * kBK, c * BN,
                         ptx::smem_u32(&ctl.full[stage]));
      }
      it += pending;
      // drain: wait (bounded) until every copy this thread issued has landed
      const uint32_t last = it;
      for (uint32_t k = (last > static_cast<uint32_t>(kStages) ? last - kStages : 0u); k < last; ++k) {
        const uint32_t stage = k % kStages, phase = (k / kStages) & 1u;
        const uint64_t t0 = ptx::globaltimer_ns();
        while (!ptx::mbar_try_wait(ptx::smem_u32(&ctl.full[stage]), phase) && ptx::globaltimer_ns() - t0 < kDrainNs) {
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = ptx::idesc_bf16_f32(kBM, BN);
      uint32_t it = 0;
      bool ok = true;
      bool issued = false;
      for (int t = 0; t < a.t_f && ok; ++t) {
        if (t > 0) {
          ok = wait_bar(ptx::smem_u32(&ctl.acc_empty), static_cast<uint32_t>((t - 1) & 1), &ctl, a.status);
          if (!ok) break;
        }
        ptx::tc_fence_after();
        for (int kb = 0; kb < KB; ++kb) {
          const uint32_t stage = it % kStages, phase = (it / kStages) & 1u;
          ok = wait_bar(ptx::smem_u32(&ctl.full[stage]), phase, &ctl, a.status);
          if (!ok) break;
          ptx::tc_fence_after();
          const uint32_t sA = ring + stage * Cfg::kStageBytes;
          const uint32_t sB = sA + Cfg::kABytes;
#pragma unroll
          for (int kk = 0; kk < kBK / 16; ++kk) {
            ptx::mma_bf16(tmem, ptx::sw128_desc(sA + kk * 32), ptx::sw128_desc(sB + kk * 32), idesc,
                          (kb | kk) != 0 ? 1u : 0u);
          }
          issued = true;
          ptx::mma_commit(ptx::smem_u32(&ctl.empty[stage]));
          ++it;
        }
        if (!ok) break;
        ptx::mma_commit(ptx::smem_u32(&ctl.acc_full));
      }
      if (!ok && issued) {
        // drain: wait (bounded) for every MMA issued so far
        ptx::mma_commit(ptx::smem_u32(&ctl.drain));
        const uint64_t t0 = ptx::globaltimer_ns();
        while (!ptx::mbar_try_wait(ptx::smem_u32(&ctl.drain), 0u) && ptx::globaltimer_ns() - t0 < kDrainNs) {
        }
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    // Warp e serves TMEM lane quarter q = warp % 4 (spins 32q..32q+31 of the tile)
    // and column group e / 4 (BN/4 replicas), 16 columns per tcgen05.ld.
    constexpr int kCW = BN / 4;
    const int e = warp - 2;
    const int q = warp & 3;
    const int col0 = (e >> 2) * kCW;
    const int i = b * kBM + q * 32 + lane;
    const bool valid = i < a.n;
    const float inv_d = a.inv_d32[i];
    const float hi = a.h32[i];
    const uint32_t lane_base = tmem + (static_cast<uint32_t>(q * 32) << 16);
    const int rbase = c * BN + col0;
    const size_t plane = static_cast<size_t>(a.r_pad) * a.n_pad;
    const RoundKeys rk = make_round_keys(a.key);
    uint32_t v[16], m[16];

    // initial state (line 2, or the given s0) -> master in TMEM and BF16 buffer 0
    for (int cc = 0; cc < kCW; cc += 16) {
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const int r = rbase + cc + k;
        float s = 0.0f;
        if (a.s0 != nullptr && valid && r < a.replicas) s = static_cast<float>(a.s0[static_cast<int64_t>(r) * a.n + i]);
        m[k] = __float_as_uint(s);
        a.S16[static_cast<size_t>(r) * a.n_pad + i] = __float2bfloat16_rn(s);
      }
      ptx::tmem_st16(lane_base + BN + col0 + cc, m);
    }
    ptx::tmem_wait_st();
    ptx::fence_proxy_async_global();
    // All epilogue warps meet on an mbarrier (release/acquire within the CTA) with a
    // bounded wait, so that a warp leaving on a timeout cannot strand the others.
    const uint32_t epi_bar = ptx::smem_u32(&ctl.epi_sync);
    auto epi_meet = [&](uint32_t phase) -> bool {
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(epi_bar);
      const bool got = wait_bar(epi_bar, phase & 1u, &ctl, a.status);
      return __all_sync(0xffffffffu, got);
    };
    bool ok = epi_meet(0);
    if (ok && e == 0 && lane == 0) ptx::st_release_gpu(a.flags + static_cast<int64_t>(b) * a.rbk + c, 1u);

    for (int t = 0; t < a.t_f && ok; ++t) {
      float inv_T = 0.0f;
      if (lane == 0) inv_T = 1.0f / static_cast<float>(a.T[t]);  // one FP64 load+convert per warp
      inv_T = __shfl_sync(0xffffffffu, inv_T, 0);
      const bool write_phi = (t == a.t_f - 1) && a.phi_out != nullptr;
      __nv_bfloat16* Snext = a.S16 + static_cast<size_t>((t + 1) & 1) * plane;
      // (A) the step's Gaussian draws do not depend on the state: generate them while
      // the tensor core computes this step's product, and park them in TMEM
      for (int cc = 0; cc < kCW; cc += 16) {
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          const int r4 = rbase + cc + 4 * g;
          const float4 z = gauss4_f32_fast(philox4x32_10_rk(
              make_uint4(static_cast<uint32_t>(r4 >> 2), static_cast<uint32_t>(t), static_cast<uint32_t>(i), a.stream),
              rk));
          v[4 * g + 0] = __float_as_uint(a.sigma_ns * z.x);
          v[4 * g + 1] = __float_as_uint(a.sigma_ns * z.y);
          v[4 * g + 2] = __float_as_uint(a.sigma_ns * z.z);
          v[4 * g + 3] = __float_as_uint(a.sigma_ns * z.w);
        }
        ptx::tmem_st16(lane_base + 2 * BN + col0 + cc, v);
      }
      ptx::tmem_wait_st();
      // (B) the update, once the product is in TMEM
      ok = __all_sync(0xffffffffu, wait_bar(ptx::smem_u32(&ctl.acc_full), static_cast<uint32_t>(t & 1), &ctl, a.status));
      if (!ok) break;
      ptx::tc_fence_after();
      for (int cc = 0; cc < kCW; cc += 16) {
        uint32_t zn[16];
        ptx::tmem_ld16(lane_base + col0 + cc, v);
        ptx::tmem_ld16(lane_base + BN + col0 + cc, m);
        ptx::tmem_ld16(lane_base + 2 * BN + col0 + cc, zn);
        ptx::tmem_wait_ld();
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const float P = __uint_as_float(v[k]) + hi;
          const float phi = fmaf(P, inv_d, __uint_as_float(zn[k]));
          const float sh = -ptx::tanh_approx(phi * inv_T);
          const float s_new = fmaf(a.alpha, sh, a.one_m_alpha * __uint_as_float(m[k]));
          m[k] = __float_as_uint(s_new);
          v[k] = __float_as_uint(phi);
        }
        if (write_phi) {  // last step of a debug run only (warp-uniform branch)
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const int r = rbase + cc + k;
            if (valid && r < a.replicas)
              a.phi_out[static_cast<int64_t>(r) * a.n + i] = static_cast<double>(__uint_as_float(v[k]));
          }
        }
        ptx::tmem_st16(lane_base + BN + col0 + cc, m);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const int r = rbase + cc + k;
          Snext[static_cast<size_t>(r) * a.n_pad + i] =
              valid ? __float2bfloat16_rn(__uint_as_float(m[k])) : __float2bfloat16_rn(0.0f);
        }
      }
      ptx::tmem_wait_st();
      ptx::tc_fence_before();
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(ptx::smem_u32(&ctl.acc_empty));
      ptx::fence_proxy_async_global();
      ok = epi_meet(static_cast<uint32_t>(t + 1));
      if (!ok) break;
      // The release store publishes every epilogue thread's state writes: they
      // happen before it through the rendezvous above (cumulativity).
      if (e == 0 && lane == 0)
        ptx::st_release_gpu(a.flags + static_cast<int64_t>(b) * a.rbk + c, static_cast<uint32_t>(t + 2));
    }
    // readout (lines 13-15): sign of the FP32 master state, zero reads as +1
    if (__all_sync(0xffffffffu, ok && !aborted(&ctl))) {
      for (int cc = 0; cc < kCW; cc += 16) {
        ptx::tmem_ld16(lane_base + BN + col0 + cc, m);
        ptx::tmem_wait_ld();
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const int r = rbase + cc + k;
          if (valid && r < a.replicas) {
            const float s = __uint_as_float(m[k]);
            a.signs[static_cast<int64_t>(r) * a.n + i] = s >= 0.0f ? int8_t(1) : int8_t(-1);
            if (a.s_out != nullptr) a.s_out[static_cast<int64_t>(r) * a.n + i] = static_cast<double>(s);
          }
        }
      }
    }
  }

  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, Cfg::kTmemCols);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// 2-D BF16 tensor map over a row-major [rows][cols] array, box = box_rows x 64.
int make_map_bf16(CUtensorMap* m, const void* base, uint64_t rows, uint64_t cols, uint32_t box_rows) {
  auto enc = get_encode_fn();
  if (enc == nullptr) return set_error(NMFA_ECUDA, "cuTensorMapEncodeTiled is unavailable");
  const cuuint64_t dims[2] = {cols, rows};
  const cuuint64_t strides[1] = {cols * 2};
  const cuuint32_t box[2] = {static_cast<cuuint32_t>(kBK), box_rows};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(NMFA_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string(r) + ")");
  return NMFA_OK;
}

int pick_bn(int32_t replicas) { return replicas <= 64 ? 64 : 128; }

template <int BN>
int launch_tc_bn(const TcProblem& pb, const RunParams& rp, const TcWorkspace& ws, cudaStream_t st) {
  using Cfg = TcCfg<BN>;
  const int nb = pb.n_pad / kBM;
  const int r_pad = (rp.replicas + BN - 1) / BN * BN;
  const int rbk = r_pad / BN;
  __nv_bfloat16* S16 = static_cast<__nv_bfloat16*>(ws.S16);
  const size_t s_bytes = 2ull * r_pad * pb.n_pad * 2;
  uint32_t* flags = reinterpret_cast<uint32_t*>(static_cast<char*>(ws.S16) + s_bytes);
  CUtensorMap tmJ, tmS;
  int rc;
  if ((rc = make_map_bf16(&tmJ, pb.Jq, pb.n_pad, pb.n_pad, kBM))) return rc;
  if ((rc = make_map_bf16(&tmS, S16, 2ull * r_pad, pb.n_pad, BN))) return rc;
  auto kern = nmfa_tc_kernel<BN>;
  if ((rc = cuda_error(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            static_cast<int>(Cfg::kSmemBytes)),
                       "tensor kernel attribute")))
    return rc;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if ((rc = cuda_error(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, Cfg::kSmemBytes),
                       "occupancy")))
    return rc;
  const int capacity = per_sm * sms;
  const int groups_per_wave = capacity / nb;
  if (groups_per_wave < 1)
    return set_error(NMFA_EUNSUPPORTED, "tensor path: n too large for one co-resident replica block");
  if ((rc = cuda_error(cudaMemsetAsync(flags, 0, sizeof(uint32_t) * nb * rbk, st), "flag reset"))) return rc;
  TcArgs a{};
  a.n = pb.n;
  a.n_pad = pb.n_pad;
  a.r_pad = r_pad;
  a.replicas = rp.replicas;
  a.t_f = rp.t_f;
  a.rbk = rbk;
  a.inv_d32 = pb.inv_d32;
  a.h32 = pb.h32;
  a.T = rp.T;
  a.sigma_ns = static_cast<float>(rp.sigma * rp.noise_sign);
  a.alpha = static_cast<float>(rp.alpha);
  a.one_m_alpha = static_cast<float>(1.0 - rp.alpha);
  a.key = make_noise_key(rp.seed);
  a.stream = rp.stream_id;
  a.s0 = rp.s0;
  a.s_out = rp.s_out;
  a.phi_out = rp.phi_out;
  a.signs = rp.signs;
  a.S16 = S16;
  a.flags = flags;
  a.status = ws.status;
  for (int c0 = 0; c0 < rbk; c0 += groups_per_wave) {
    a.c_offset = c0;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(nb, std::min(groups_per_wave, rbk - c0), 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = Cfg::kSmemBytes;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if ((rc = cuda_error(cudaLaunchKernelEx(&cfg, kern, tmJ, tmS, a), "tensor kernel launch"))) return rc;
    count_launch();
  }
  return NMFA_OK;
}

}  // namespace

int tc_workspace_bytes(const TcProblem& pb, int32_t replicas, int64_t* bytes) {
  const int bn = pick_bn(replicas);
  const int64_t r_pad = (replicas + bn - 1) / bn * bn;
  const int64_t nb = pb.n_pad / kBM;
  *bytes = 2 * r_pad * pb.n_pad * 2 + (nb * (r_pad / bn) * 4 + 255) / 256 * 256;
  return NMFA_OK;
}

int launch_tc(const TcProblem& pb, const RunParams& rp, const TcWorkspace& ws, cudaStream_t st) {
  if (pb.fp8) return set_error(NMFA_EUNSUPPORTED, "FP8-J tensor path is not available in this build");
  if (pb.n_pad % kBM != 0) return set_error(NMFA_EINVAL, "tensor path: n_pad must be a multiple of 128");
  return pick_bn(rp.replicas) == 64 ? launch_tc_bn<64>(pb, rp, ws, st) : launch_tc_bn<128>(pb, rp, ws, st);
}


// ----------------------------------------------------------------------------
// Scratch without allocation, for nmfa_run_device_noalloc.
//
// The tensor path's scratch (the two BF16 state buffers and the per-tile epoch
// flags) normally lives in memory the problem handle allocates on demand.  Callers
// that must not allocate device memory get it from this file-scope array instead.
// It is created when the GPU loads this library's device code and stays there
// until the process exits, on every GPU that loads the library.  Host code cannot
// use the symbol itself as a device address, so its address is looked up once per
// device (with that device current) and cached.
// ----------------------------------------------------------------------------
namespace {
constexpr size_t kStaticScratchBytes = size_t(16) << 20;  // 16 MiB
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];
}  // namespace

int tc_static_scratch(void** ptr, size_t* bytes) {
  static std::mutex mu;
  static void* addr[128] = {};
  int dev = 0;
  int rc = cuda_error(cudaGetDevice(&dev), "cudaGetDevice");
  if (rc) return rc;
  if (dev < 0 || dev >= 128) return set_error(NMFA_EUNSUPPORTED, "device ordinal out of range for static scratch");
  std::lock_guard<std::mutex> g(mu);
  if (addr[dev] == nullptr) {
    void* p = nullptr;
    rc = cuda_error(cudaGetSymbolAddress(&p, g_static_scratch), "cudaGetSymbolAddress(static scratch)");
    if (rc) return rc;
    addr[dev] = p;
  }
  *ptr = addr[dev];
  *bytes = kStaticScratchBytes;
  return NMFA_OK;
}

int launch_tc_static_scratch(const TcProblem& pb, const RunParams& rp, int32_t* status, cudaStream_t st) {
  int64_t need = 0;
  int rc = tc_workspace_bytes(pb, rp.replicas, &need);
  if (rc) return rc;
  if (need > static_cast<int64_t>(kStaticScratchBytes))
    return set_error(NMFA_EINVAL, "nmfa_run_device_noalloc: this size needs " + std::to_string(need) +
                                      " bytes of scratch, more than the 16 MiB static buffer");
  void* p = nullptr;
  size_t bytes = 0;
  if ((rc = tc_static_scratch(&p, &bytes))) return rc;
  TcWorkspace ws{};
  ws.S16 = p;
  ws.status = status;
  ws.bytes = need;
  return launch_tc(pb, rp, ws, st);  // clears the epoch flags before the kernel runs
}

}  // namespace nmfa
