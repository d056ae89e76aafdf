// k_tc.cu -- the tcgen05 tensor-core path of NMFA (BF16 J and S, FP32 accumulation).
//
// One persistent launch runs all t_f steps of Algorithm 1 for a batch of replicas
// (one run, or a ragged batch of runs of different instances).  The coupling
// product of the field update over all replicas is the GEMM P = J S (J: n x n,
// S: n x R).  The replicas of a run are split into groups of BN (64, 128 or 256); a
// group's output is tiled by row blocks of 128 spins, and each (group, row block)
// item is owned by one tile pipeline for the group's whole run.  A pipeline is a
// TMA warp, an MMA warp and BN / 8 epilogue warps (16 for BN = 256); a CTA holds
// one pipeline for BN = 128 or 256 and two independent ones for BN = 64 (one CTA per
// SM), and walks the work list the host planned for it:
//   - the TMA warp streams 128-deep K slices of J's row block and of S's replica
//     block into a ring of shared-memory slots (128-byte swizzle); the J slices of
//     a step start before the step's state is published, and each S slice as soon
//     as the row block that wrote it has published the step, in a fixed K order that
//     starts with the tile's own slice (signalled by a shared-memory barrier that the
//     tile's own epilogue warps complete; the other slices by the row blocks' epoch
//     flags);
//   - the MMA warp issues tcgen05.mma (M = 128, N = BN, K = 16; one elected lane of
//     the converged warp) into one of two TMEM accumulators, releasing ring slots
//     and the accumulator with tcgen05.commit;
//   - the epilogue warps draw the next step's noise (Philox/Box-Muller, independent
//     of the state) while the tensor core works and write h_i + sigma z d_i into
//     the next accumulator, so that the product lands on it; once the accumulator
//     is complete they read it with tcgen05.ld and finish the step: division by
//     d_i, -tanh(Phi/T_t) and the alpha-mix into the FP32 master state, which stays
//     in TMEM for the whole run; the new state is written in BF16 to the next of
//     two global S buffers (L2-resident) and published by each warp's release
//     increment of the tile's epoch counter.
// Step t+1's slices of row block b' are loaded only after tile b' has published
// step t, which realises the synchronous update of Algorithm 1 (every Phi from the
// old state) without a grid-wide barrier: only the pipelines of one group depend on
// one another.  After the last step the signs are read out from the FP32 master
// state; for integer problems one more product of J with the sign vectors gives the
// Eq. (1) energies exactly.
//
// Every wait (mbarrier or flag) is bounded by a 2-second wall-clock limit (20 s for
// the flag waits of a group's first step, which may follow groups scheduled before
// it); on
// expiry the pipeline records NMFA's timeout status, drains its own TMA copies and
// MMAs, and the CTA frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "nmfa_device.cuh"
#include "nmfa_internal.h"
#include "tc_ptx.cuh"

namespace nmfa {

namespace {

constexpr int kBM = 128;               // spins per tile (TMEM lanes)
constexpr int kBK = 64;                // K atom: 64 BF16 = one 128-byte swizzle row
constexpr int kColsPerWarp = 32;
// Ring slots of a 128-deep K slice (two swizzle atoms): eight MMAs per slot.  An
// M = 128, N <= 128 tcgen05.mma costs its issuing warp about as long as its own tensor
// work, so the handshake per slot (full-barrier wait, commit) is amortised over
// eight MMAs rather than four (measured on GB300 with the noise draws running: ~77
// instead of ~101 clocks per MMA against 64 of tensor work).  Slot layout:
// [A atom 0][A atom 1][B atom 0][B atom 1].
constexpr int kAtoms = 2;
constexpr int kKSlot = kAtoms * kBK;
constexpr int kMaxStages = 4;
constexpr uint32_t kABytes = kBM * 128;  // one A (J) atom: 128 rows x 128 bytes
// Geometry per tile width BN (replicas per tile, the MMA's N: 64, 128 or 256).
//   Epilogue warps: each serves one TMEM lane quarter and 32 replica columns, so a
//   tile takes BN / 8 of them (16 for 128-replica tiles, 8 for 64).
//   One CTA per SM: a kernel that allocates TMEM is given one CTA per SM by the
//   occupancy rules, which the cooperative launch follows.  A 128-replica CTA runs
//   one tile pipeline (TMA warp, MMA warp, 16 epilogue warps) with a ring of 3
//   slots of 64 KB.  A 64-replica CTA runs two independent pipelines (2 x 10 warps),
//   each with its own ring of 2 slots of 48 KB, barriers, work list and half of
//   the TMEM: a 64-replica tile's products are short, and the second pipeline's
//   MMAs fill the time the first spends in its epilogue and state exchange.
//   TMEM columns of a pipeline (from its base): accumulators [0, BN) and
//   [BN, 2 BN) (step g uses g % 2), FP32 master state [2 BN, 3 BN).
//   A 256-replica CTA (for runs whose 128-replica tiles would need more than one
//   wave of the grid) has one pipeline of 16 epilogue warps with 64 columns each, a
//   ring of 2 slots of 96 KB, and a single accumulator [0, 256) beside the master
//   state [256, 512): its MMAs (N = 256) run near the full tensor rate, and each
//   step's bias is written into the accumulator after the update has read it.
//   A CTA PAIR (PAIR = true, 128 replicas) is a cluster of two CTAs that share one
//   cta_group::2 MMA of M = 256: the pair owns two adjacent row blocks (256 spins) of
//   a group, each CTA its own block (its TMEM lanes, its epilogue warps, its J rows)
//   and half of the group's replicas of every S slice (the B operand), so each SM
//   lands 48 KB of operands per 128-deep K slice instead of 64 KB, and the tensor
//   core reads 96 instead of 128 bytes per clock from each SM's shared memory (at
//   the full MMA rate).  Ring of 4 slots of 48 KB; the even CTA issues the MMAs.
//   FP8 (F8 = true, 64, 128 or 256 replicas, one CTA per tile): J is stored in E4M3 (in
//   the byte order (k0, k2, k1, k3) within each 4-value group); its slices go by TMA
//   into a 2-buffer staging ring of 16 KB (128 rows x 128 K bytes) and are written as
//   BF16 into the slot's A operand (the MMA stays kind::f16 with both operands BF16)
//   by eight converter warps, one 16-row part of every slice each (the tile's 8
//   epilogue warps then cover twice the columns of the BF16 form: more warps would
//   put six on one scheduler, whose register file then allows 80 registers a thread
//   instead of 96); the slot's full barrier then also waits for every converter
//   warp.
template <int BN, bool PAIR = false, bool F8 = false>
struct TcShape {
  static constexpr bool kDoubleAcc = BN != 256;     // two accumulators (bias written ahead)
  // epilogue warps of 32 columns (64- and 128-replica tiles) or 64 (256-replica
  // tiles); with FP8 couplings twice as wide (8 warps), leaving room for 8 converter
  // warps in the same 18 warps and 96 registers a thread
  static constexpr int kColsPerWarp = (F8 && BN == 256) ? 128 : (BN == 256 || (F8 && BN == 128)) ? 64 : 32;
  static constexpr int kEpiWarps = 4 * BN / kColsPerWarp;
  static constexpr int kSubs = (BN == 64 && !PAIR && !F8) ? 2 : 1;  // tile pipelines per CTA
  static constexpr int kConvWarps = F8 ? 8 : 0;  // FP8 -> BF16 converter warps
  static constexpr int kSubWarps = 2 + kEpiWarps + kConvWarps;  // warps per pipeline
  static constexpr int kThreads = 32 * kSubWarps * kSubs;
  static constexpr int kBRows = PAIR ? BN / 2 : BN;  // replica rows of each B slice in this CTA
  // ring slots per pipeline (the FP8 64-replica CTA has one pipeline, room for four)
  static constexpr int kStages = PAIR ? 4 : (BN == 128 ? 3 : ((BN == 64 && F8) ? 4 : 2));
  static constexpr uint32_t kBAtomBytes = kBRows * 128;  // one B (S) atom: kBRows rows x 128 bytes
  static constexpr uint32_t kStageBytes = kAtoms * (kABytes + kBAtomBytes);
  static constexpr int kMmaM = PAIR ? 2 * kBM : kBM;
  static constexpr uint32_t kRingBytes = kStages * kStageBytes;
  static constexpr uint32_t kStgBytes = kBM * kKSlot;  // one E4M3 slice: 128 rows x 128 K bytes
  static constexpr int kStgStages = 2;
  static constexpr size_t kSmemBytes =
      static_cast<size_t>(kSubs) * kRingBytes + (F8 ? kStgStages * kStgBytes : 0u) + 1024;
  static constexpr uint32_t kTmemCols = 512;  // allocated once per CTA
  static constexpr uint32_t kSubCols = kTmemCols / kSubs;
  static constexpr uint32_t kColAcc1 = kDoubleAcc ? BN : 0;
  static constexpr uint32_t kColMaster = kDoubleAcc ? 2 * BN : BN;
  static_assert(kStages <= kMaxStages, "ring slots");
  static_assert(kColMaster + BN <= kSubCols, "TMEM columns");
  static_assert(kEpiWarps * kColsPerWarp == 4 * BN, "every (quarter, column) pair once");
  static_assert(kSmemBytes <= 227 * 1024, "shared memory");
  static_assert(!PAIR || BN == 128, "CTA pairs take 128-replica tiles");
  static_assert(!F8 || !PAIR, "FP8 couplings take one-CTA tiles");
};
constexpr uint64_t kTimeoutNs = 2000000000ull;
// A pipeline that reaches a new group early waits for the group's other pipelines to
// finish the groups scheduled before it; that first wait gets a longer bound.
constexpr uint64_t kStartTimeoutNs = 20000000000ull;
constexpr uint64_t kDrainNs = 200000000ull;

// One replica block of one instance: the tile pipelines that exchange state every step.
struct __align__(64) TcGroup {
  CUtensorMap tmJ;        // BF16 J of the instance, [n_pad][n_pad], box 64 x 128
  CUtensorMap tmS;        // this group's state buffers, [2 * bn][n_pad], box 64 x bn
  const float* inv_d32;
  const float* h32;
  const double* T;
  const double* s0;       // instance-level (replica-major, n per replica) or null
  double* s_out;
  double* phi_out;
  int8_t* signs;
  __nv_bfloat16* S16;     // [2][bn][n_pad]
  uint32_t* flags;        // [nb] epoch counters
  int64_t* e2h;           // [bn] 2H of the group's replicas, accumulated (zeroed every launch)
  uint32_t* e_done;       // epilogue warps that have added their part of 2H (zeroed every launch)
  double* energy;         // instance-level [replicas] or null
  int64_t* energy_i64;    // instance-level [replicas] or null
  int32_t energy_pass;    // 1: the run ends with the energy product J s~ (see epilogue_item)
  int32_t n, n_pad, bn, replicas, r0, t_f;
  float sigma_ns, alpha, one_m_alpha;
  uint32_t seed_lo, seed_hi, stream;
};
struct TcItem {
  int32_t group, b;
};

struct SharedCtl {
  uint64_t full[kMaxStages];
  uint64_t empty[kMaxStages];
  uint64_t acc_full;
  // The step's accumulator holds its bias (epilogue -> MMA).  Step g uses
  // bias_ready[g % 2]: every epilogue warp arrives for step g + 1 before it waits for
  // step g's product, so with one barrier a fast warp's arrival for g + 1 could
  // complete step g's phase before a slow warp has written step g's bias.  Between two
  // uses of the same barrier each warp waits for acc_full of the step in between,
  // which implies the earlier phase completed.
  uint64_t bias_ready[2];
  // Completes once per publication of this pipeline's tile state that the producer
  // copies from (publications 1 .. t_f + energy pass of an item; every epilogue warp
  // arrives after its state writes and proxy fence): the producer copies the tile's
  // own K slice on it without a round trip through the epoch counter in L2.  Arrivals
  // and waits pair one to one, so the barrier is never more than one phase ahead.
  uint64_t own_pub;
  // CTA pairs: completes once per publication of the PEER CTA's tile state (its
  // epilogue warps arrive from the other CTA), so each CTA copies the pair's other
  // row block without a round trip through that block's epoch counter.
  uint64_t pair_pub;
  // FP8: staged E4M3 slice landed (TMA) / converted by all of its tasks
  uint64_t stg_full[2];
  uint64_t stg_empty[2];
  uint64_t drain;
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

// Bounded mbarrier wait; false if the run is being aborted.  `cluster`: acquire at
// cluster scope (barriers that the peer CTA of a pair arrives on).
__device__ __forceinline__ bool try_bar(uint32_t bar, uint32_t parity, bool cluster) {
  return cluster ? ptx::mbar_try_wait_cluster(bar, parity) : ptx::mbar_try_wait(bar, parity);
}
__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity, SharedCtl* ctl, int32_t* status,
                                         uint64_t limit_ns = kTimeoutNs, bool cluster = false) {
  if (try_bar(bar, parity, cluster)) return true;
  const uint64_t t0 = ptx::globaltimer_ns();
  while (true) {
    if (try_bar(bar, parity, cluster)) return true;
    if (aborted(ctl)) return false;
    if (ptx::globaltimer_ns() - t0 > limit_ns) {
      raise_abort(ctl, status);
      return false;
    }
  }
}

// Row blocks of a group seen published at the current step: lane l holds bit j for
// row block l + 32 j (a group has at most 304 row blocks, two pipelines on each of
// 152 SMs, so j < 10).
__device__ __forceinline__ bool block_seen(uint32_t seen, int k) {
  return (__shfl_sync(0xffffffffu, seen, k & 31) >> (k >> 5)) & 1u;
}

// Wait (bounded) until row block k of the group has published step counter `need`.
// Each poll reads every counter not yet seen, one acquire load per row block, so one
// round trip to L2 also finds the blocks the producer will need next.  The warp
// barrier and the proxy fence after the poll order the owning lane's acquire before
// the copies that the elected lane issues from that block's state.
__device__ __forceinline__ bool wait_block(const uint32_t* f0, int nb, int k, uint32_t need, int lane,
                                           uint32_t& seen, SharedCtl* ctl, int32_t* status, bool first_step) {
  if (block_seen(seen, k)) return true;
  const uint64_t limit_ns = first_step ? kStartTimeoutNs : kTimeoutNs;
  const uint64_t t0 = ptx::globaltimer_ns();
  while (true) {
    uint32_t bit = 1u;
    for (int rb = lane; rb < nb; rb += 32, bit <<= 1)
      if (!(seen & bit) && ptx::ld_acquire_gpu(f0 + rb) >= need) seen |= bit;
    __syncwarp();
    if (block_seen(seen, k)) {
      ptx::fence_proxy_async_global();
      return true;
    }
    int stop = 0;
    if (lane == 0) {
      if (aborted(ctl)) {
        stop = 1;
      } else if (ptx::globaltimer_ns() - t0 > limit_ns) {
        raise_abort(ctl, status);
        stop = 1;
      }
    }
    if (__shfl_sync(0xffffffffu, stop, 0)) return false;
  }
}

// ---------------------------------------------------------------- FP8 conversion
// A staged E4M3 slice of fill f (128 rows x 128 K values, 128-byte swizzle) becomes
// the BF16 A operand of ring slot f % kStages (two 128-byte-swizzle atoms of 64 K
// values).  Each converter warp takes every fill in order and converts its share of
// the slice's kConvParts parts of 16 rows, so it waits on the staging barriers and
// on the slots' empty barriers in fill order and never one phase ahead.  The
// producer stages fill f's slice before it waits for the ring slot (the copy
// overlaps the MMAs still reading the slot); the converter waits for the slot to be
// released before it writes, then arrives on the staging buffer's empty barrier and
// on the slot's full barrier (one arrival per converter warp each).
constexpr uint32_t kConvParts = 8;

// Rows 16 part .. 16 part + 15 of a staged slice -> BF16 atoms.  A 16-byte access is
// served 8 lanes at a time, so each group of 8 lanes takes one 16-value chunk c
// (K values 16c .. 16c + 15) of 8 consecutive rows: their 8 row swizzles (r mod 8)
// put both the loads and the stores of the group on 8 distinct 16-byte bank groups.
// Lane l converts chunk l / 8 + 4 (u / 2) of row 16 part + l % 8 + 8 (u % 2),
// u = 0 .. 3, ILP chunks at a time.
template <int ILP>
__device__ __forceinline__ void convert_part(uint32_t src, uint32_t dst, uint32_t part, int lane) {
#pragma unroll
  for (int u0 = 0; u0 < 4; u0 += ILP) {
    uint4 v[ILP];
#pragma unroll
    for (int u = 0; u < ILP; ++u) {
      const uint32_t r = part * 16u + static_cast<uint32_t>(lane & 7) + 8u * ((u0 + u) & 1);
      const uint32_t c = static_cast<uint32_t>(lane >> 3) + 4u * ((u0 + u) >> 1);
      v[u] = ptx::ld_shared_v4(src + r * 128u + ((c ^ (r & 7u)) << 4));
    }
#pragma unroll
    for (int u = 0; u < ILP; ++u) {
      const uint32_t r = part * 16u + static_cast<uint32_t>(lane & 7) + 8u * ((u0 + u) & 1);
      const uint32_t c = static_cast<uint32_t>(lane >> 3) + 4u * ((u0 + u) >> 1);
      const uint32_t sw = r & 7u;
      uint4 lo, hi;  // BF16 values 16c .. 16c + 7 and 16c + 8 .. 16c + 15
      ptx::e4m3x4p_to_bf16x2x2(v[u].x, lo.x, lo.y);
      ptx::e4m3x4p_to_bf16x2x2(v[u].y, lo.z, lo.w);
      ptx::e4m3x4p_to_bf16x2x2(v[u].z, hi.x, hi.y);
      ptx::e4m3x4p_to_bf16x2x2(v[u].w, hi.z, hi.w);
      // atom c / 4 holds K 64 (c / 4) .. + 63; the chunk's 16 values fill chunks
      // 2 (c % 4) and 2 (c % 4) + 1 of row r there
      const uint32_t row = dst + (c >> 2) * kABytes + r * 128u;
      const uint32_t c0 = 2u * (c & 3u);
      ptx::st_shared_v4(row + ((c0 ^ sw) << 4), lo);
      ptx::st_shared_v4(row + (((c0 + 1u) ^ sw) << 4), hi);
    }
  }
}

// Converter warp cw's share of fill f: parts cw, cw + kConvWarps, ...
template <int BN>
__device__ __forceinline__ bool conv_fill(SharedCtl* ctl, int32_t* status, uint32_t ring, uint32_t stg, uint32_t f,
                                          int cw, int lane) {
  using Shape = TcShape<BN, false, true>;
  constexpr uint32_t kStages = static_cast<uint32_t>(Shape::kStages);
  const uint32_t jb = f & 1u, st = f % kStages;
  if (!__all_sync(0xffffffffu, wait_bar(ptx::smem_u32(&ctl->stg_full[jb]), (f >> 1) & 1u, ctl, status))) return false;
  if (!__all_sync(0xffffffffu, wait_bar(ptx::smem_u32(&ctl->empty[st]), ((f / kStages) & 1u) ^ 1u, ctl, status)))
    return false;
#pragma unroll 1
  for (uint32_t part = static_cast<uint32_t>(cw); part < kConvParts; part += Shape::kConvWarps)
    convert_part<4>(stg + jb * Shape::kStgBytes, ring + st * Shape::kStageBytes, part, lane);
  ptx::fence_proxy_async_shared();
  __syncwarp();
  if (lane == 0) {
    ptx::mbar_arrive(ptx::smem_u32(&ctl->stg_empty[jb]));
    ptx::mbar_arrive(ptx::smem_u32(&ctl->full[st]));
  }
  return true;
}

// The tensor maps live in global memory (written by an earlier kernel); make the
// tensormap proxy see those writes before the first copy that uses them.
__device__ __forceinline__ void acquire_tensormap(const void* m) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(m))
               : "memory");
}

// Barrier that tells the MMA issuer step g's bias is in place: one per accumulator.
template <int BN>
__device__ __forceinline__ uint32_t bias_bar(SharedCtl* ctl, uint32_t g) {
  return ptx::smem_u32(&ctl->bias_ready[TcShape<BN>::kDoubleAcc ? (g & 1u) : 0u]);
}

// Tells the MMA issuer that this warp's part of step g's bias is written: on the
// CTA's own barrier, or (the odd CTA of a pair) on the even CTA's, which issues the
// pair's MMAs.
template <int BN>
__device__ __forceinline__ void arrive_bias(SharedCtl* ctl, uint32_t g, bool remote) {
  const uint32_t bar = bias_bar<BN>(ctl, g);
  if (remote)
    ptx::mbar_arrive_cluster(ptx::mapa_shared(bar, 0u));
  else
    ptx::mbar_arrive(bar);
}

// (A) the bias of one step, h_i + sigma z d_i, written into the accumulator the step
// will use (the Gaussian draws do not depend on the state, so with two accumulators
// this runs while the tensor core still computes the previous step), then signalled
// to the MMA issuer.
template <int BN, bool F8 = false>
__device__ __forceinline__ void write_bias(int t, uint32_t g, uint32_t lane_base, int col0, int rbase, int i,
                                           uint32_t stream, const RoundKeys& rk, float sigma_ns, float dd, float hi,
                                           int lane, SharedCtl* ctl, bool remote) {
  const uint32_t acc = lane_base + ((g & 1u) ? TcShape<BN, false, F8>::kColAcc1 : 0u);
  uint32_t v[16];
#pragma unroll 1
  for (int cc = 0; cc < TcShape<BN, false, F8>::kColsPerWarp; cc += 16) {
#pragma unroll
    for (int gq = 0; gq < 4; ++gq) {
      const int r4 = rbase + cc + 4 * gq;
      const float4 z = gauss4_f32_fast(philox4x32_10_rk(
          make_uint4(static_cast<uint32_t>(r4 >> 2), static_cast<uint32_t>(t), static_cast<uint32_t>(i), stream), rk));
      v[4 * gq + 0] = __float_as_uint(fmaf(sigma_ns * z.x, dd, hi));
      v[4 * gq + 1] = __float_as_uint(fmaf(sigma_ns * z.y, dd, hi));
      v[4 * gq + 2] = __float_as_uint(fmaf(sigma_ns * z.z, dd, hi));
      v[4 * gq + 3] = __float_as_uint(fmaf(sigma_ns * z.w, dd, hi));
    }
    ptx::tmem_st16(acc + col0 + cc, v);
  }
  ptx::tmem_wait_st();
  ptx::tc_fence_before();
  __syncwarp();
  if (lane == 0) arrive_bias<BN>(ctl, g, remote);
}

// (A') the accumulator start of the energy product: 2 h_i, no noise.
template <int BN, bool F8 = false>
__device__ __forceinline__ void write_energy_bias(uint32_t g, uint32_t lane_base, int col0, float hi, int lane,
                                                  SharedCtl* ctl, bool remote) {
  const uint32_t acc = lane_base + ((g & 1u) ? TcShape<BN, false, F8>::kColAcc1 : 0u);
  uint32_t v[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = __float_as_uint(2.0f * hi);
#pragma unroll 1
  for (int cc = 0; cc < TcShape<BN, false, F8>::kColsPerWarp; cc += 16) ptx::tmem_st16(acc + col0 + cc, v);
  ptx::tmem_wait_st();
  ptx::tc_fence_before();
  __syncwarp();
  if (lane == 0) arrive_bias<BN>(ctl, g, remote);
}

// Publication of this tile's state (every epilogue warp, after its state writes and
// proxy fence): the CTA's own producer (own_pub), the peer CTA's producer of a pair
// (its pair_pub), then the tile's epoch counter for every other tile of the group.
template <bool PAIR>
__device__ __forceinline__ void publish(SharedCtl* ctl, uint32_t* my_flag, bool to_producers, uint32_t crank) {
  if (to_producers) {
    ptx::mbar_arrive(ptx::smem_u32(&ctl->own_pub));
    if constexpr (PAIR) ptx::mbar_arrive_cluster(ptx::mapa_shared(ptx::smem_u32(&ctl->pair_pub), crank ^ 1u));
  }
  ptx::red_release_gpu_add(my_flag, 1u);
}

// (C) Energy readout (Eq. 1) of one warp's 32 spins x 32 replicas.  The accumulator
// of the energy product started at 2 h_i, so it holds P_i = 2 h_i + sum_j J_ij s~_j,
// and sum_i s~_i P_i = 2 H(s~) because J is symmetric with zero diagonal.  Every
// partial sum is an integer below 2^24, so the FP32 accumulator holds P_i exactly and
// the sums over spins are taken in integers.  Each warp adds its part to the group's
// 2H sums; the warp that adds the group's last part (`parts` in all) writes the
// energies.  Kept out of line: it runs once per item and its registers would
// otherwise weigh on the step loop.
__device__ __noinline__ void energy_readout(const TcGroup* __restrict__ g, uint32_t acc, uint32_t master, int col0,
                                            int rbase, bool valid, int lane, uint32_t parts) {
  const int R = g->replicas;
  int mine = 0;  // lane c: this warp's part of 2H for column col0 + c
#pragma unroll 1
  for (int cc = 0; cc < kColsPerWarp; cc += 16) {
    uint32_t pa[16], ms[16];
    ptx::tmem_ld16(acc + col0 + cc, pa);
    ptx::tmem_ld16(master + col0 + cc, ms);
    ptx::tmem_wait_ld();
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int r = rbase + cc + k;
      int v = 0;
      if (valid && r < R) {
        const int pi = __float2int_rn(__uint_as_float(pa[k]));
        v = __uint_as_float(ms[k]) >= 0.0f ? pi : -pi;
      }
      const int sum = __reduce_add_sync(0xffffffffu, v);  // 32 spins, |sum| < 2^29
      if (lane == cc + k) mine = sum;
    }
  }
  if (rbase + lane < R)
    atomicAdd(reinterpret_cast<unsigned long long*>(g->e2h + col0 + lane),
              static_cast<unsigned long long>(static_cast<long long>(mine)));
  // each warp fences its additions before counting itself done
  __threadfence();
  __syncwarp();
  uint32_t prev = 0;
  if (lane == 0) prev = atomicAdd(g->e_done, 1u);
  prev = __shfl_sync(0xffffffffu, prev, 0);
  if (prev + 1 == parts) {
    __threadfence();
    for (int c = lane; c < g->bn; c += 32) {
      const int r = g->r0 + c;
      if (r < R) {
        const long long e2 = static_cast<long long>(atomicAdd(reinterpret_cast<unsigned long long*>(g->e2h + c), 0ull));
        const long long H = e2 / 2;  // 2H is even: sum_i s~_i (J s~)_i counts every pair twice
        if (g->energy_i64 != nullptr) g->energy_i64[r] = H;
        if (g->energy != nullptr) g->energy[r] = static_cast<double>(H);
      }
    }
  }
}

// Epilogue warps' work for one item (one 128-spin tile of one group), from the
// initial state through t_f steps to the readout.  Epilogue warp e of a pipeline is
// physical warp e + QOFF (mod 4), which may access TMEM lane quarter
// q = (e + QOFF) % 4 (spins 32q..32q+31 of the tile); it serves that quarter and
// column group e / 4 (32 replicas), 16 columns per tcgen05.ld.  `gstep` counts the CTA's steps across items
// (the parity of the accumulator barriers).  Returns false on abort.
template <int BN, int QOFF, bool PAIR, bool F8 = false>
__device__ __forceinline__ bool epilogue_item(const TcGroup* __restrict__ g, int b, int e, int lane, uint32_t tmem,
                                              SharedCtl* ctl, int32_t* status, uint32_t& gstep, uint32_t crank) {
  const bool remote_bias = PAIR && crank != 0u;
  using Shape = TcShape<BN, false, F8>;
  constexpr int kCW = Shape::kColsPerWarp;
  constexpr bool kDouble = Shape::kDoubleAcc;
  constexpr uint32_t kColAcc1 = Shape::kColAcc1, kColMaster = Shape::kColMaster;
  const int q = (e + QOFF) & 3;
  const uint32_t lane_base = tmem + (static_cast<uint32_t>(q * 32) << 16);
  const int n = g->n, n_pad = g->n_pad, t_f = g->t_f, R = g->replicas;
  const int col0 = (e >> 2) * kCW;
  const int i = b * kBM + q * 32 + lane;
  const bool valid = i < n;
  const float inv_d = g->inv_d32[i];
  const float hi = g->h32[i];
  const int rbase = g->r0 + col0;  // replica index (of the instance) of column col0
  const size_t plane = static_cast<size_t>(BN) * n_pad;
  const RoundKeys rk = make_round_keys(NoiseKey{g->seed_lo, g->seed_hi});
  const float sigma_ns = g->sigma_ns, alpha = g->alpha, oma = g->one_m_alpha;
  const int energy_pass = g->energy_pass;
  const uint32_t stream = g->stream;
  const double* T = g->T;
  double* phi_out = g->phi_out;
  __nv_bfloat16* S16 = g->S16;
  uint32_t* my_flag = g->flags + b;
  uint32_t m[16];

  // the initial state (zero, or the given s0) -> master in TMEM and BF16 buffer 0
  const double* s0 = g->s0;
#pragma unroll 1
  for (int cc = 0; cc < kCW; cc += 16) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int r = rbase + cc + k;
      float s = 0.0f;
      if (s0 != nullptr && valid && r < R) s = static_cast<float>(s0[static_cast<int64_t>(r) * n + i]);
      m[k] = __float_as_uint(s);
      S16[static_cast<size_t>(col0 + cc + k) * n_pad + i] = __float2bfloat16_rn(s);
    }
    ptx::tmem_st16(lane_base + kColMaster + col0 + cc, m);
  }
  ptx::tmem_wait_st();
  // Publication: every epilogue warp adds 1 to its tile's epoch counter with a
  // release reduction once its lanes' state writes are done (the warp barrier orders
  // the lanes' writes before lane 0's release), so the counter reaches
  // (epilogue warps) * (t + 1) when the whole tile of state S_t is visible.
  ptx::fence_proxy_async_global();
  __syncwarp();
  if (lane == 0) publish<PAIR>(ctl, my_flag, t_f + energy_pass >= 1, crank);

  // Row constants: with d_i > 0 the accumulator starts at h_i + sigma z d_i so that
  // acc / d_i = (h_i + sum_j J_ij s_j) / d_i + sigma z; a spin with d_i = 0 (no
  // couplings, no field) starts at sigma z and is scaled by 1.
  const float dd = inv_d > 0.0f ? 1.0f / inv_d : 1.0f;
  const float sc = inv_d > 0.0f ? inv_d : 1.0f;
  // (A) the bias of step t: the Gaussian draws do not depend on the state, so they
  // are generated while the tensor core still computes the previous step
  if (t_f > 0)
    write_bias<BN, F8>(0, gstep, lane_base, col0, rbase, i, stream, rk, sigma_ns, dd, hi, lane, ctl, remote_bias);

  for (int t = 0; t < t_f; ++t, ++gstep) {
    float inv_T = 0.0f;
    if (lane == 0) inv_T = 1.0f / static_cast<float>(T[t]);  // one FP64 load+convert per warp
    inv_T = __shfl_sync(0xffffffffu, inv_T, 0);
    __nv_bfloat16* Snext = S16 + static_cast<size_t>((t + 1) & 1) * plane;
    // the next step's bias goes into the other accumulator (read last two steps ago)
    if constexpr (kDouble) {
      if (t + 1 < t_f)
        write_bias<BN, F8>(t + 1, gstep + 1, lane_base, col0, rbase, i, stream, rk, sigma_ns, dd, hi, lane, ctl,
                       remote_bias);
      else if (energy_pass)
        write_energy_bias<BN, F8>(gstep + 1, lane_base, col0, hi, lane, ctl, remote_bias);
    }
    // (B) the update, once the product is in TMEM
    if (!__all_sync(0xffffffffu, wait_bar(ptx::smem_u32(&ctl->acc_full), gstep & 1u, ctl, status))) return false;
    ptx::tc_fence_after();
    const uint32_t acc = lane_base + ((gstep & 1u) ? kColAcc1 : 0u);
    const bool write_phi = (t == t_f - 1) && phi_out != nullptr;
    // the last step hands the energy product the sign vector s~ instead of s
    const bool write_sign = energy_pass && t == t_f - 1;
#pragma unroll
    for (int cc = 0; cc < kCW; cc += 16) {
      uint32_t pa[16], ms[16];
      ptx::tmem_ld16(acc + col0 + cc, pa);
      ptx::tmem_ld16(lane_base + kColMaster + col0 + cc, ms);
      ptx::tmem_wait_ld();
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const float phi = __uint_as_float(pa[k]) * sc;
        const float sh = -ptx::tanh_approx(phi * inv_T);
        const float s_new = fmaf(alpha, sh, oma * __uint_as_float(ms[k]));
        ms[k] = __float_as_uint(s_new);
        pa[k] = __float_as_uint(phi);
      }
      if (write_phi) {  // last step of a debug run only (warp-uniform branch)
        if constexpr (BN == 64) {
          double* po = phi_out + static_cast<int64_t>(rbase + cc) * n + i;
          const int rmax = valid ? R - (rbase + cc) : 0;  // columns k < rmax are replicas of the run
#pragma unroll
          for (int k = 0; k < 16; ++k)
            if (k < rmax) po[k * n] = static_cast<double>(__uint_as_float(pa[k]));
        } else {
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const int r = rbase + cc + k;
            if (valid && r < R) phi_out[static_cast<int64_t>(r) * n + i] = static_cast<double>(__uint_as_float(pa[k]));
          }
        }
      }
      ptx::tmem_st16(lane_base + kColMaster + col0 + cc, ms);
      if (!write_sign) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          Snext[static_cast<size_t>(col0 + cc + k) * n_pad + i] =
              valid ? __float2bfloat16_rn(__uint_as_float(ms[k])) : __float2bfloat16_rn(0.0f);
        }
      } else {  // kept apart: a select inside the loop above slows every step
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const float sv = __uint_as_float(ms[k]) >= 0.0f ? 1.0f : -1.0f;
          Snext[static_cast<size_t>(col0 + cc + k) * n_pad + i] = valid ? __float2bfloat16_rn(sv) : __float2bfloat16_rn(0.0f);
        }
      }
    }
    ptx::tmem_wait_st();
    ptx::fence_proxy_async_global();
    __syncwarp();
    // publication t + 1 (the producers copy it only if another step follows)
    if (lane == 0) publish<PAIR>(ctl, my_flag, t + 2 <= t_f + energy_pass, crank);
    if constexpr (!kDouble) {
      // one accumulator: the next step's bias goes in once this step's product has
      // been read (the draws then overlap the other tiles' publication and the copies)
      if (t + 1 < t_f)
        write_bias<BN, F8>(t + 1, gstep + 1, lane_base, col0, rbase, i, stream, rk, sigma_ns, dd, hi, lane, ctl,
                       remote_bias);
      else if (energy_pass)
        write_energy_bias<BN, F8>(gstep + 1, lane_base, col0, hi, lane, ctl, remote_bias);
    }
  }
  // sign readout of Algorithm 1: sign of the FP32 master state, zero reads as +1
  if (!__all_sync(0xffffffffu, !aborted(ctl))) return false;
  int8_t* signs = g->signs;
  double* s_out = g->s_out;
#pragma unroll 1
  for (int cc = 0; cc < kCW; cc += 16) {
    ptx::tmem_ld16(lane_base + kColMaster + col0 + cc, m);
    ptx::tmem_wait_ld();
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int r = rbase + cc + k;
      if (valid && r < R) {
        const float s = __uint_as_float(m[k]);
        signs[static_cast<int64_t>(r) * n + i] = s >= 0.0f ? int8_t(1) : int8_t(-1);
        if (s_out != nullptr) s_out[static_cast<int64_t>(r) * n + i] = static_cast<double>(s);
      }
    }
  }
  // (C) energy readout (Eq. 1), after the energy product of the last step's signs
  if (energy_pass) {
    if (!__all_sync(0xffffffffu, wait_bar(ptx::smem_u32(&ctl->acc_full), gstep & 1u, ctl, status))) return false;
    ptx::tc_fence_after();
    // 32 columns per call: parts = tiles x BN / 32 per group
#pragma unroll 1
    for (int c2 = 0; c2 < kCW; c2 += kColsPerWarp)
      energy_readout(g, lane_base + ((gstep & 1u) ? kColAcc1 : 0u), lane_base + kColMaster, col0 + c2, rbase + c2,
                     valid, lane, static_cast<uint32_t>(n_pad / kBM) * static_cast<uint32_t>(BN / 8));
    ++gstep;
  }
  return true;
}

// One tile pipeline of the persistent kernel: its TMA warp (lw 0), MMA warp (lw 1) and
// epilogue warps (lw 2..), its control block, ring slots, TMEM columns and work list
// (plan slot SUB * gridDim.x + blockIdx.x; for CTA pairs the cluster's slot, shared by
// both CTAs).  SUB is a template argument so that the control block's shared-memory
// address stays a constant.
//
// K order: every one-CTA tile of a group sweeps the group's K slices (row blocks)
// starting at its own row block b and wrapping, whatever its width (64, 128 or 256
// replicas, BF16- or FP8-stored J), so the FP32 sums of every output, and with them the
// results, do not depend on the width.  The two tiles of a CTA pair share one MMA and
// therefore one order, starting at the pair's even row block (b & ~1): the pair's odd
// tile sums in another order than a one-CTA tile would, so CTA-pair runs agree with
// one-CTA runs to the BF16 path's rounding, not bit for bit.  (The shared order for
// every variant cost 4-5 % on small and mid-size groups, whose odd row blocks then
// waited for their partner's slice, which comes through L2, before their own.)
template <int BN, int SUB, bool PAIR, bool F8>
__device__ __forceinline__ void run_pipeline(const TcGroup* __restrict__ groups, const TcItem* __restrict__ items,
                                             const int32_t* __restrict__ first, int32_t* status, SharedCtl* ctl_all,
                                             uint32_t ring_base, uint32_t tmem_base, int warp, int lane) {
  using Shape = TcShape<BN, PAIR, F8>;
  constexpr int kEpiWarps = Shape::kEpiWarps;
  constexpr int kSubWarps = Shape::kSubWarps;
  constexpr int kStages = Shape::kStages;
  constexpr uint32_t kStageBytes = Shape::kStageBytes, kBAtomBytes = Shape::kBAtomBytes;
  constexpr uint32_t kColAcc1 = Shape::kColAcc1;
  SharedCtl& ctl = ctl_all[SUB];
  const int lw = warp - SUB * kSubWarps;
  const uint32_t crank = PAIR ? ptx::cluster_ctarank() : 0u;
  const int slot = PAIR ? static_cast<int>(blockIdx.x >> 1)
                        : SUB * static_cast<int>(gridDim.x) + static_cast<int>(blockIdx.x);
  const int w_begin = first[slot], w_end = first[slot + 1];
  const uint32_t ring = ring_base + static_cast<uint32_t>(SUB) * Shape::kRingBytes;
  const uint32_t tmem = tmem_base + static_cast<uint32_t>(SUB) * Shape::kSubCols;
  // FP8 staging ring (after the operand ring; 1024-aligned like it)
  const uint32_t stg_base = ring_base + static_cast<uint32_t>(Shape::kSubs) * Shape::kRingBytes;

  if (lw == 0) {
    // ------------------------------------------------------------ TMA producer
    // Per step: claim the first ring slots and start their J slices at once (J
    // does not depend on the previous step), then issue each slot's S slice once its
    // row block has published the step's state (the own block: own_pub; the pair's
    // other block: pair_pub; the others: their epoch counters), and stream the rest
    // of the step.  The whole warp runs the loop; one elected lane issues each copy.
    // In a pair the even CTA's full barriers count both CTAs' copies (the odd CTA's
    // copies complete on them); each CTA waits on its own empty barriers, which the
    // pair's MMA commits signal in both CTAs.
    const uint32_t full0 = ptx::smem_u32(&ctl.full[0]), empty0 = ptx::smem_u32(&ctl.empty[0]);
    const uint32_t full0_lead = PAIR ? ptx::mapa_shared(full0, 0u) : full0;
    const bool lead = crank == 0u;
    uint32_t stage = 0, phase = 0;  // next ring slot to fill
    uint32_t filled = 0;            // ring slots whose copies were issued (for the drain)
    uint32_t staged = 0;            // FP8: staging copies issued (for the drain)
    uint32_t own_pubs = 0;          // own_pub (and pair_pub) phases completed by earlier items
    bool ok = true;
    auto load = [&](uint32_t dst, const void* tm, int x, int y, uint32_t st) {
      if (PAIR && !lead)
        ptx::tma_load_2d_pair_warp(dst, tm, x, y, full0_lead + 8u * st);
      else
        ptx::tma_load_2d_warp(dst, tm, x, y, full0 + 8u * st);
    };
    const uint32_t stg_full0 = ptx::smem_u32(&ctl.stg_full[0]), stg_empty0 = ptx::smem_u32(&ctl.stg_empty[0]);
    for (int w = w_begin; w < w_end && ok; ++w) {
      const TcItem item = items[w];
      const TcGroup* g = groups + item.group;
      const int b = PAIR ? 2 * item.b + static_cast<int>(crank) : item.b;  // this CTA's row block
      const int n_pad = g->n_pad, nb = n_pad / kBM, bn = g->bn, steps = g->t_f + g->energy_pass;
      const void* tmJ = &g->tmJ;
      const void* tmS = &g->tmS;
      const uint32_t* gflags = g->flags;
      // bytes that complete one slot's full barrier: both CTAs' copies for a pair; for
      // FP8 only the S copies (the converter warps write the J operand and arrive)
      const uint32_t stage_tx = (PAIR ? 2u : 1u) * kAtoms *
                                ((F8 ? 0u : kABytes) + static_cast<uint32_t>(PAIR ? bn / 2 : bn) * 128u);
      // the J slice of fill `fill` into ring slot `st`: BF16 straight into the slot, or
      // (FP8) the E4M3 slice into the staging buffer the converter warps read
      auto load_j = [&](int ks, uint32_t st, uint32_t fill) -> bool {
        if constexpr (F8) {
          const uint32_t jb = fill & 1u;
          if (!__all_sync(0xffffffffu, wait_bar(stg_empty0 + 8u * jb, ((fill >> 1) & 1u) ^ 1u, &ctl, status)))
            return false;
          ptx::mbar_arrive_expect_tx_warp(stg_full0 + 8u * jb, Shape::kStgBytes);
          ptx::tma_load_2d_warp(stg_base + jb * Shape::kStgBytes, tmJ, ks * kKSlot, b * kBM, stg_full0 + 8u * jb);
          ++staged;
        } else {
#pragma unroll
          for (int a = 0; a < kAtoms; ++a) load(ring + st * kStageBytes + a * kABytes, tmJ, ks * kKSlot + a * kBK, b * kBM, st);
        }
        return true;
      };
      const int brow = PAIR ? static_cast<int>(crank) * (bn / 2) : 0;  // this CTA's replica rows of S
      const int KB = n_pad / kKSlot;  // ring slots per step (= row blocks)
      const int kslice_base = (PAIR ? (b & ~1) : b) % KB;
      if (lane == 0) {
        acquire_tensormap(tmJ);
        acquire_tensormap(tmS);
        ptx::tma_prefetch_desc(tmJ);
        ptx::tma_prefetch_desc(tmS);
      }
      __syncwarp();
      const int pre = KB < kStages ? KB : kStages;
      for (int t = 0; t < steps && ok; ++t) {
        const int sy = (t & 1) * bn + brow;
        const uint32_t claim_stage = stage;
        int claimed = 0;
        int ks = kslice_base;  // K slice of loop index kb
        for (int kb = 0; kb < pre; ++kb) {
          // FP8: the E4M3 slice is staged before the slot is free (the conversion
          // tasks wait for the slot)
          if constexpr (F8) {
            ok = load_j(ks, stage, filled);
            if (!ok) break;
          }
          ok = __all_sync(0xffffffffu, wait_bar(empty0 + 8u * stage, phase ^ 1u, &ctl, status));
          if (!ok) break;
          if (lead) ptx::mbar_arrive_expect_tx_warp(full0 + 8u * stage, stage_tx);
          if constexpr (!F8) load_j(ks, stage, filled);
          ++claimed;
          ++filled;
          if (++stage == kStages) {
            stage = 0;
            phase ^= 1u;
          }
          if (++ks == KB) ks = 0;
        }
        // Each S half is copied as soon as its own row block has published the step, in
        // the fixed K order (so the FP32 sums keep one order): the tile's own slice and
        // (pairs) the pair's other slice on shared-memory barriers, the others on their
        // epoch counters, so that the MMAs on early blocks overlap the wait for a late one.
        const uint32_t need = static_cast<uint32_t>(kEpiWarps * (t + 1));
        uint32_t seen = 0;
        {
          uint32_t st = claim_stage;
          int ks2 = kslice_base;
          for (int kb = 0; kb < claimed; ++kb) {  // (issued on abort too, so that the barriers complete)
            if (ok && ks2 == b) {
              // the tile's own slice, published by this pipeline's epilogue: own_pub
              // completes once per publication the producer copies from
              ok = __all_sync(0xffffffffu, wait_bar(ptx::smem_u32(&ctl.own_pub), (own_pubs + t) & 1u, &ctl, status,
                                                    t == 0 ? kStartTimeoutNs : kTimeoutNs));
              if (ok) ptx::fence_proxy_async_global();
            } else if (PAIR && ok && ks2 == (b ^ 1)) {
              // the pair's other row block, published by the peer CTA's epilogue
              ok = __all_sync(0xffffffffu, wait_bar(ptx::smem_u32(&ctl.pair_pub), (own_pubs + t) & 1u, &ctl, status,
                                                    t == 0 ? kStartTimeoutNs : kTimeoutNs, true));
              if (ok) ptx::fence_proxy_async_global();
            } else if (ok) {
              ok = wait_block(gflags, nb, ks2, need, lane, seen, &ctl, status, t == 0);
            }
#pragma unroll
            for (int a = 0; a < kAtoms; ++a)
              load(ring + st * kStageBytes + kAtoms * kABytes + a * kBAtomBytes, tmS, ks2 * kKSlot + a * kBK, sy, st);
            if (++st == kStages) st = 0;
            if (++ks2 == KB) ks2 = 0;
          }
        }
        if (!ok) break;
        for (int kb = pre; kb < KB; ++kb) {
          if constexpr (F8) {
            ok = load_j(ks, stage, filled);
            if (!ok) break;
          }
          ok = __all_sync(0xffffffffu, wait_bar(empty0 + 8u * stage, phase ^ 1u, &ctl, status));
          if (!ok) break;
          const uint32_t sA = ring + stage * kStageBytes;
          if (lead) ptx::mbar_arrive_expect_tx_warp(full0 + 8u * stage, stage_tx);
          if constexpr (!F8) load_j(ks, stage, filled);
          ok = wait_block(gflags, nb, ks, need, lane, seen, &ctl, status, t == 0);
#pragma unroll
          for (int a = 0; a < kAtoms; ++a)
            load(sA + kAtoms * kABytes + a * kBAtomBytes, tmS, ks * kKSlot + a * kBK, sy, stage);
          ++filled;
          if (++stage == kStages) {
            stage = 0;
            phase ^= 1u;
          }
          if (++ks == KB) ks = 0;
          if (!ok) break;
        }
      }
      own_pubs += static_cast<uint32_t>(steps);
    }
    if (!ok) {
      // drain: wait (bounded) until every copy issued into the last ring slots has
      // landed.  A pair's copies complete on the even CTA's full barriers, so the odd
      // CTA waits for its own slots to be released by the MMA commits instead.
      const uint32_t last = filled;
      if constexpr (F8) {
        // the staged E4M3 copies of the last fills (their barriers complete on landing)
        for (uint32_t k = (staged > 2u ? staged - 2u : 0u); k < staged; ++k) {
          const uint64_t t0 = ptx::globaltimer_ns();
          while (!ptx::mbar_try_wait(stg_full0 + 8u * (k & 1u), (k >> 1) & 1u) && ptx::globaltimer_ns() - t0 < kDrainNs) {
          }
        }
      }
      for (uint32_t k = (last > static_cast<uint32_t>(kStages) ? last - kStages : 0u); k < last; ++k) {
        const uint32_t st = k % kStages, ph = (k / kStages) & 1u;
        const uint64_t t0 = ptx::globaltimer_ns();
        if (PAIR && !lead) {
          while (!ptx::mbar_try_wait(empty0 + 8u * st, ph) && ptx::globaltimer_ns() - t0 < kDrainNs) {
          }
        } else {
          while (!ptx::mbar_try_wait(full0 + 8u * st, ph) && ptx::globaltimer_ns() - t0 < kDrainNs) {
          }
        }
      }
    }
  } else if (lw == 1) {
    // ------------------------------------------------------------ MMA issuer
    // The whole warp runs the loop and one elected lane issues each tcgen05.mma and
    // commit.  The ring position is carried as (stage, phase) counters and the
    // shared-memory descriptors are formed once and advanced by adding to their
    // start-address field (32 bytes per K = 16 step, one atom or slot further on; the
    // field cannot carry out of its 14 bits because shared addresses stay below 256 KB).
    // A pair's MMAs (M = 256 across both CTAs) are issued by the even CTA alone; its
    // commits arrive on the barriers of both CTAs.
    if (PAIR && crank != 0u) return;
    uint32_t stage = 0, phase = 0, gstep = 0;
    bool ok = true;
    bool issued = false;
    const uint64_t desc0 = ptx::sw128_desc(ring);
    constexpr uint64_t kDescStage = kStageBytes >> 4, kDescA = kABytes >> 4, kDescB = (kAtoms * kABytes) >> 4,
                       kDescBAtom = kBAtomBytes >> 4, kDescK = 32 >> 4;
    const uint32_t full0 = ptx::smem_u32(&ctl.full[0]), empty0 = ptx::smem_u32(&ctl.empty[0]);
    for (int w = w_begin; w < w_end && ok; ++w) {
      const TcGroup* g = groups + items[w].group;
      const int KB = g->n_pad / kKSlot, steps = g->t_f + g->energy_pass;
      // every group of a plan has the kernel's tile width: N = BN
      constexpr uint32_t idesc = ptx::idesc_bf16_f32(Shape::kMmaM, BN);
      for (int t = 0; t < steps && ok; ++t, ++gstep) {
        // the epilogue has written this step's bias (h + sigma z d) into the
        // accumulator the step uses (in both CTAs of a pair); the product
        // accumulates onto it
        ok = __all_sync(0xffffffffu, wait_bar(bias_bar<BN>(&ctl, gstep),
                                              Shape::kDoubleAcc ? ((gstep >> 1) & 1u) : (gstep & 1u), &ctl, status,
                                              kTimeoutNs, PAIR));
        if (!ok) break;
        ptx::tc_fence_after();
        const uint32_t acc = tmem + ((gstep & 1u) ? kColAcc1 : 0u);
        for (int kb = 0; kb < KB; ++kb) {
          // the stage's TMA copies completed on its full barrier (async proxy to async proxy)
          ok = __all_sync(0xffffffffu, wait_bar(full0 + 8u * stage, phase, &ctl, status));
          if (!ok) break;
          const uint64_t da = desc0 + kDescStage * stage;
#pragma unroll
          for (int a = 0; a < kAtoms; ++a) {
#pragma unroll
            for (int kk = 0; kk < kBK / 16; ++kk) {
              if constexpr (PAIR)
                ptx::mma_bf16_pair_warp(acc, da + kDescA * a + kDescK * kk, da + kDescB + kDescBAtom * a + kDescK * kk,
                                        idesc);
              else
                ptx::mma_bf16_warp(acc, da + kDescA * a + kDescK * kk, da + kDescB + kDescBAtom * a + kDescK * kk,
                                   idesc);
            }
          }
          issued = true;
          if constexpr (PAIR)
            ptx::mma_commit_pair_warp(empty0 + 8u * stage, 0x3);
          else
            ptx::mma_commit_warp(empty0 + 8u * stage);
          if (++stage == kStages) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
        if constexpr (PAIR)
          ptx::mma_commit_pair_warp(ptx::smem_u32(&ctl.acc_full), 0x3);
        else
          ptx::mma_commit_warp(ptx::smem_u32(&ctl.acc_full));
      }
    }
    if (!ok && issued) {
      // drain: wait (bounded) for every MMA issued so far
      if constexpr (PAIR)
        ptx::mma_commit_pair_warp(ptx::smem_u32(&ctl.drain), 0x1);
      else
        ptx::mma_commit_warp(ptx::smem_u32(&ctl.drain));
      const uint64_t t0 = ptx::globaltimer_ns();
      while (!ptx::mbar_try_wait(ptx::smem_u32(&ctl.drain), 0u) && ptx::globaltimer_ns() - t0 < kDrainNs) {
      }
    }
  } else if (F8 && lw >= 2 + kEpiWarps) {
    // ------------------------------------------------------------ FP8 converters
    if constexpr (F8) {
      uint32_t total = 0;  // ring fills of this pipeline
      for (int w = w_begin; w < w_end; ++w) {
        const TcGroup* g = groups + items[w].group;
        total += static_cast<uint32_t>((g->t_f + g->energy_pass) * (g->n_pad / kKSlot));
      }
      for (uint32_t f = 0; f < total; ++f)
        if (!conv_fill<BN>(&ctl, status, ring, stg_base, f, lw - 2 - kEpiWarps, lane)) break;
    }
  } else {
    // ------------------------------------------------------------ epilogue
    // epilogue warp e (physical warp e + 2 + SUB * kSubWarps) serves column group
    // e / 4 and the TMEM lane quarter that warp may access; over the pipeline's
    // warps each (quarter, column group) pair occurs once
    const int e = lw - 2;
    uint32_t gstep = 0;
    bool ok = true;
    for (int w = w_begin; w < w_end && ok; ++w) {
      const TcItem item = items[w];
      const TcGroup* g = groups + item.group;
      const int b = PAIR ? 2 * item.b + static_cast<int>(crank) : item.b;
      ok = epilogue_item<BN, (2 + SUB * kSubWarps) & 3, PAIR, F8>(g, b, e, lane, tmem, &ctl, status, gstep, crank);
    }
  }
}

template <int BN, bool PAIR = false, bool F8 = false>
__global__ void __launch_bounds__(TcShape<BN, PAIR, F8>::kThreads, 1)
nmfa_tc_kernel(const TcGroup* __restrict__ groups, const TcItem* __restrict__ items, const int32_t* __restrict__ first,
               int32_t* status) {
  using Shape = TcShape<BN, PAIR, F8>;
  constexpr int kEpiWarps = Shape::kEpiWarps;
  constexpr int kSubs = Shape::kSubs, kSubWarps = Shape::kSubWarps;
  constexpr int kStages = Shape::kStages;
  constexpr uint32_t kTmemCols = Shape::kTmemCols;
  extern __shared__ __align__(1024) uint8_t smem_dyn[];
  __shared__ SharedCtl ctl_all[kSubs];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t ring_base = (ptx::smem_u32(smem_dyn) + 1023u) & ~1023u;

  if (threadIdx.x == 0) {
    for (int p = 0; p < kSubs; ++p) {
      SharedCtl& c = ctl_all[p];
      for (int s = 0; s < kStages; ++s) {
        // FP8: the producer's arrival (S bytes) and one arrival per converter warp
        ptx::mbar_init(ptx::smem_u32(&c.full[s]), 1 + Shape::kConvWarps);
        ptx::mbar_init(ptx::smem_u32(&c.empty[s]), 1);
      }
      for (int j = 0; j < 2; ++j) {
        ptx::mbar_init(ptx::smem_u32(&c.stg_full[j]), 1);
        ptx::mbar_init(ptx::smem_u32(&c.stg_empty[j]), F8 ? Shape::kConvWarps : 1);
      }
      ptx::mbar_init(ptx::smem_u32(&c.acc_full), 1);
      // a pair's MMA issuer waits for the bias of both CTAs' epilogue warps
      ptx::mbar_init(ptx::smem_u32(&c.bias_ready[0]), (PAIR ? 2 : 1) * kEpiWarps);
      ptx::mbar_init(ptx::smem_u32(&c.bias_ready[1]), (PAIR ? 2 : 1) * kEpiWarps);
      ptx::mbar_init(ptx::smem_u32(&c.own_pub), kEpiWarps);
      ptx::mbar_init(ptx::smem_u32(&c.pair_pub), kEpiWarps);
      ptx::mbar_init(ptx::smem_u32(&c.drain), 1);
      c.abort_flag = 0;
    }
    ptx::fence_mbar_init();
  }
  if (warp == 1) {
    if constexpr (PAIR) {
      // one warp of each CTA of the pair allocates together
      ptx::tmem_alloc_pair<kTmemCols>(ptx::smem_u32(&ctl_all[0].tmem_slot));
      ptx::tmem_relinquish_pair();
    } else {
      ptx::tmem_alloc<kTmemCols>(ptx::smem_u32(&ctl_all[0].tmem_slot));
      ptx::tmem_relinquish();
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  // a pair's CTAs start once both have initialised their barriers and allocated
  if constexpr (PAIR) ptx::cluster_sync();
  ptx::tc_fence_after();
  const uint32_t tmem_base = ctl_all[0].tmem_slot;

  if constexpr (kSubs == 1) {
    run_pipeline<BN, 0, PAIR, F8>(groups, items, first, status, ctl_all, ring_base, tmem_base, warp, lane);
  } else {
    if (warp < kSubWarps)
      run_pipeline<BN, 0, PAIR, F8>(groups, items, first, status, ctl_all, ring_base, tmem_base, warp, lane);
    else
      run_pipeline<BN, 1, PAIR, F8>(groups, items, first, status, ctl_all, ring_base, tmem_base, warp, lane);
  }

  ptx::tc_fence_before();
  __syncthreads();
  // neither CTA of a pair leaves (or frees its tensor memory) while the pair's MMAs
  // may still read its shared memory or write its tensor memory: every wait above is
  // bounded, so both CTAs reach this barrier
  if constexpr (PAIR) ptx::cluster_sync();
  if (warp == 1) {
    ptx::tc_fence_after();
    if constexpr (PAIR)
      ptx::tmem_dealloc_pair<kTmemCols>(tmem_base);
    else
      ptx::tmem_dealloc<kTmemCols>(tmem_base);
  }
}

// Copies a block of plan bytes (group descriptors, items, CTA offsets) from the
// kernel's parameter space to device memory: no host-pinned buffer and no
// allocation, so it can be recorded in a CUDA graph.
constexpr int kUploadBytes = 30720;
struct TcUpload {
  uint32_t bytes;
  uint32_t pad[3];
  uint4 data[kUploadBytes / 16];
};
__global__ void tc_upload_kernel(const __grid_constant__ TcUpload u, uint4* dst) {
  for (uint32_t k = threadIdx.x; k < u.bytes / 16; k += blockDim.x) dst[k] = u.data[k];
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

// Co-resident scheduling units of the persistent grid for one tile variant: CTAs
// (one per SM), or for CTA pairs the clusters of two that fit at once.
// 2-D E4M3 (one byte per value) tensor map over a row-major [rows][cols] array, box =
// 128 rows x 128 bytes with the 128-byte swizzle (the converter warps' staging layout).
int make_map_u8(CUtensorMap* m, const void* base, uint64_t rows, uint64_t cols) {
  auto enc = get_encode_fn();
  if (enc == nullptr) return set_error(NMFA_ECUDA, "cuTensorMapEncodeTiled is unavailable");
  const cuuint64_t dims[2] = {cols, rows};
  const cuuint64_t strides[1] = {cols};
  const cuuint32_t box[2] = {static_cast<cuuint32_t>(kKSlot), static_cast<cuuint32_t>(kBM)};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(NMFA_ECUDA, "cuTensorMapEncodeTiled (E4M3) failed (" + std::to_string(r) + ")");
  return NMFA_OK;
}

template <int BN, bool PAIR, bool F8>
int co_resident_units_t(int* capacity) {
  static int cached = -1;
  if (cached < 0) {
    using Shape = TcShape<BN, PAIR, F8>;
    int rc;
    if ((rc = cuda_error(cudaFuncSetAttribute(nmfa_tc_kernel<BN, PAIR, F8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              static_cast<int>(Shape::kSmemBytes)),
                         "tensor kernel attribute")))
      return rc;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if constexpr (PAIR) {
      cudaLaunchConfig_t cfg{};
      cfg.gridDim = dim3(static_cast<unsigned>(2 * (sms / 2)), 1, 1);
      cfg.blockDim = dim3(Shape::kThreads, 1, 1);
      cfg.dynamicSmemBytes = Shape::kSmemBytes;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = 2;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      int clusters = 0;
      if ((rc = cuda_error(cudaOccupancyMaxActiveClusters(&clusters, nmfa_tc_kernel<BN, PAIR, F8>, &cfg),
                           "cluster occupancy")))
        return rc;
      cached = std::min(clusters, sms / 2);
    } else {
      if ((rc = cuda_error(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, nmfa_tc_kernel<BN, PAIR, F8>,
                                                                         Shape::kThreads, Shape::kSmemBytes),
                           "occupancy")))
        return rc;
      // never more CTAs on an SM than its TMEM holds (each allocates kTmemCols of 512)
      per_sm = std::min(per_sm, static_cast<int>(512 / Shape::kTmemCols));
      cached = per_sm * sms;
    }
  }
  *capacity = cached;
  return NMFA_OK;
}
int co_resident_units(int bn, bool pair, bool f8, int* capacity) {
  if (pair) return co_resident_units_t<128, true, false>(capacity);
  if (f8)
    return bn == 256  ? co_resident_units_t<256, false, true>(capacity)
           : bn == 64 ? co_resident_units_t<64, false, true>(capacity)
                      : co_resident_units_t<128, false, true>(capacity);
  return bn == 64 ? co_resident_units_t<64, false, false>(capacity)
                  : bn == 256 ? co_resident_units_t<256, false, false>(capacity)
                              : co_resident_units_t<128, false, false>(capacity);
}
// Tile pipelines per scheduling unit.
int tc_subs(int bn, bool pair, bool f8) { return (bn == 64 && !pair && !f8) ? TcShape<64>::kSubs : 1; }
// Work-list slots of the co-resident grid: tile pipelines, or CTA pairs.
int co_resident_slots(int bn, bool pair, bool f8, int* slots) {
  int units = 0;
  const int rc = co_resident_units(bn, pair, f8, &units);
  if (rc) return rc;
  *slots = units * tc_subs(bn, pair, f8);
  return NMFA_OK;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

// Default tile width of a run.  64 replicas per tile for runs of at most 64
// replicas; also for problems of n_pad <= 1024 whose 128-replica tiles would leave
// more than half the SMs without one: their J stays in L2, so narrower tiles on twice
// the SMs take less operand stream per SM (measured on GB300, 200-step runs, ms:
// n = 512, R = 1024: 1.13 -> 0.89; n = 1024, R = 1024: 1.39 -> 1.20; R = 512: 1.38 ->
// 1.23).  Larger problems keep 128 (n = 4096, R = 256: 3.03 against 3.27; n = 8192,
// R = 128: 6.82 against 7.95, where each extra replica block re-reads a J that does not
// fit in L2).  Results do not depend on the width.
int tc_pick_bn(int32_t replicas, int32_t n_pad) {
  if (replicas <= 64) return 64;
  static int sms = 0;
  if (sms == 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
      sms = v;
  }
  const int64_t tiles128 = static_cast<int64_t>(n_pad / kBM) * ((replicas + 127) / 128);
  if (n_pad <= 1024 && sms > 0 && 2 * tiles128 <= sms) return 64;
  // 256 replicas per tile when 128-replica tiles would need more than one wave of
  // the grid (one CTA per SM) and a step has at least 16 K slices: half the tiles,
  // each streaming J once for twice the replicas with MMAs of N = 256.  Their single
  // accumulator puts the next step's noise draws after the update, which only a long
  // enough product hides (200-step runs, ms, 256 against 128: n = 2048, R = 2048:
  // 3.77 / 4.33; n = 4096, R = 1024: 6.04 / 6.90; n = 8192, R = 512: 11.7 / 13.9;
  // but n = 1536, R = 4096: 6.57 / 5.32).
  if (sms > 0 && tiles128 > sms && replicas > 128 && n_pad >= 2048) return 256;
  return 128;
}

// Whether 128-replica tiles of an n_pad problem CAN run as CTA pairs (one
// cta_group::2 MMA of M = 256 per pair of adjacent row blocks): the row blocks pair
// up (n_pad a multiple of 256) and the group's pairs fit on the grid at once.  Pairs
// are an option (NMFA_BATCH_PAIR128), not the default: measured on GB300 (SK n = 2000,
// 1024 replicas) they run 10.43 against 9.71 ms per run, because the MMA phase is
// paced by MMA instruction issue (about 100 clocks per instruction under the epilogue
// warps' noise draws, whether the instruction covers 128 or 256 rows), not by the
// operand bytes the pair halves.  Results do not depend on it.
bool tc_use_pair(int bn, int32_t n_pad) {
  if (bn != 128 || n_pad % (2 * kBM) != 0) return false;
  int clusters = 0;
  if (co_resident_units(128, true, false, &clusters) != NMFA_OK) {
    cudaGetLastError();
    return false;
  }
  return n_pad / (2 * kBM) <= clusters;
}

// ---------------------------------------------------------------------------
// Planning: every job (instance run) is split into groups of bn replicas; every
// group needs nb = n_pad/128 co-resident CTAs for its whole run.  Groups are placed
// on the persistent grid's CTA slots by list scheduling (longest first, on the nb
// slots that free up earliest), so each CTA walks its items in start order and any
// CTA waiting for a group's peers waits only on groups that started earlier: no
// cycle of waits can form.
// ---------------------------------------------------------------------------
int tc_plan_bytes(const TcJob* jobs, int32_t count, int64_t* bytes) {
  if (count < 1) return set_error(NMFA_EINVAL, "empty plan");
  int capacity = 0;  // tile pipelines (or CTA pairs) of the co-resident grid
  const bool pair = jobs[0].pair, f8 = jobs[0].pb.fp8;
  int rc = co_resident_slots(jobs[0].bn, pair, f8, &capacity);
  if (rc) return rc;
  size_t ngroups = 0, nitems = 0, flags = 0, state = 0;
  for (int j = 0; j < count; ++j) {
    const int bn = jobs[j].bn;
    const int nb = jobs[j].pb.n_pad / kBM;
    if (bn != jobs[0].bn || jobs[j].pair != pair || jobs[j].pb.fp8 != f8)
      return set_error(NMFA_EINVAL, "one plan takes one tile variant");
    if (f8 && pair) return set_error(NMFA_EINVAL, "FP8 couplings take one-CTA tiles");
    if (pair && nb % 2 != 0) return set_error(NMFA_EINVAL, "CTA pairs need an even number of row blocks");
    const int units = pair ? nb / 2 : nb;
    if (units > capacity)
      return set_error(NMFA_EUNSUPPORTED, "tensor path: n too large for one co-resident replica block");
    const int groups = (jobs[j].rp.replicas + bn - 1) / bn;
    ngroups += groups;
    nitems += static_cast<size_t>(groups) * units;
    flags += static_cast<size_t>(groups) * nb;
    state += static_cast<size_t>(groups) * 2 * bn * jobs[j].pb.n_pad * 2;
  }
  // cleared every launch: epoch flags, then per group one done-counter and bn 2H sums
  const size_t cleared = align_up(flags * 4, 256) + align_up(ngroups * 4, 256) +
                         align_up(ngroups * static_cast<size_t>(jobs[0].bn) * 8, 256);
  *bytes = static_cast<int64_t>(align_up(ngroups * sizeof(TcGroup), 256) + align_up(nitems * sizeof(TcItem), 256) +
                                align_up((static_cast<size_t>(capacity) + 1) * 4, 256) + cleared + state);
  return NMFA_OK;
}

int tc_build_plan(const TcJob* jobs, int32_t count, void* ws, int64_t ws_bytes, int32_t* status, TcPlan* plan,
                  bool withhold_tile) {
  if (count < 1) return set_error(NMFA_EINVAL, "empty plan");
  const bool pair = jobs[0].pair, f8 = jobs[0].pb.fp8;
  int ctas = 0;  // scheduling units: CTAs, or CTA pairs
  int rc = co_resident_units(jobs[0].bn, pair, f8, &ctas);
  if (rc) return rc;
  const int subs = tc_subs(jobs[0].bn, pair, f8);
  // scheduler slot s is pipeline s / ctas of unit s % ctas: every unit's first
  // pipeline fills before any second one
  const int capacity = ctas * subs;
  int64_t need = 0;
  if ((rc = tc_plan_bytes(jobs, count, &need))) return rc;
  if (need > ws_bytes) return set_error(NMFA_EINVAL, "tensor path: workspace too small");
  struct G {
    int job, c, nb;
    double dur;
  };
  std::vector<G> gl;
  size_t nitems = 0, nflags = 0;
  for (int j = 0; j < count; ++j) {
    const int bn = jobs[j].bn, nb = jobs[j].pb.n_pad / kBM;
    const int units = pair ? nb / 2 : nb;  // work items (tiles, or pairs of tiles) of a group
    const int groups = (jobs[j].rp.replicas + bn - 1) / bn;
    const int steps = jobs[j].rp.t_f + (tc_fuses_energy(jobs[j].pb, jobs[j].rp) ? 1 : 0);
    for (int c = 0; c < groups; ++c) {
      gl.push_back({j, c, units, static_cast<double>(steps) * (2.0 * nb + 8.0)});
      nitems += units;
      nflags += nb;
    }
  }
  char* base = static_cast<char*>(ws);
  const size_t off_items = align_up(gl.size() * sizeof(TcGroup), 256);
  const size_t off_first = off_items + align_up(nitems * sizeof(TcItem), 256);
  const size_t off_flags = off_first + align_up((static_cast<size_t>(capacity) + 1) * 4, 256);
  const size_t off_done = off_flags + align_up(nflags * 4, 256);
  const size_t off_e2h = off_done + align_up(gl.size() * 4, 256);
  const size_t off_state = off_e2h + align_up(gl.size() * static_cast<size_t>(jobs[0].bn) * 8, 256);
  // group descriptors
  plan->host.assign(off_flags, 0);
  plan->group_job.resize(gl.size());
  TcGroup* hg = reinterpret_cast<TcGroup*>(plan->host.data());
  size_t flag_pos = 0, state_pos = off_state;
  std::vector<uint32_t*> gflags(gl.size());
  for (size_t k = 0; k < gl.size(); ++k) {
    const TcJob& jb = jobs[gl[k].job];
    plan->group_job[k] = gl[k].job;
    TcGroup& g = hg[k];
    const int bn = jb.bn;
    g.n = jb.pb.n;
    g.n_pad = jb.pb.n_pad;
    g.bn = bn;
    g.replicas = jb.rp.replicas;
    g.r0 = gl[k].c * bn;
    g.t_f = jb.rp.t_f;
    g.inv_d32 = jb.pb.inv_d32;
    g.h32 = jb.pb.h32;
    g.T = jb.rp.T;
    g.s0 = jb.rp.s0;
    g.s_out = jb.rp.s_out;
    g.phi_out = jb.rp.phi_out;
    g.signs = jb.rp.signs;
    g.sigma_ns = static_cast<float>(jb.rp.sigma * jb.rp.noise_sign);
    g.alpha = static_cast<float>(jb.rp.alpha);
    g.one_m_alpha = static_cast<float>(1.0 - jb.rp.alpha);
    g.seed_lo = static_cast<uint32_t>(jb.rp.seed);
    g.seed_hi = static_cast<uint32_t>(jb.rp.seed >> 32);
    g.stream = jb.rp.stream_id;
    g.flags = reinterpret_cast<uint32_t*>(base + off_flags) + flag_pos;
    flag_pos += g.n_pad / kBM;
    g.energy_pass = tc_fuses_energy(jb.pb, jb.rp) ? 1 : 0;
    g.e_done = reinterpret_cast<uint32_t*>(base + off_done) + k;
    g.e2h = reinterpret_cast<int64_t*>(base + off_e2h) + k * static_cast<size_t>(bn);
    g.energy = g.energy_pass ? jb.rp.energy : nullptr;
    g.energy_i64 = g.energy_pass ? jb.rp.energy_i64 : nullptr;
    g.S16 = reinterpret_cast<__nv_bfloat16*>(base + state_pos);
    state_pos += static_cast<size_t>(2) * bn * g.n_pad * 2;
    if ((rc = f8 ? make_map_u8(&g.tmJ, jb.pb.Jq, g.n_pad, g.n_pad) : make_map_bf16(&g.tmJ, jb.pb.Jq, g.n_pad, g.n_pad, kBM)))
      return rc;
    // a pair's CTAs each load half of the group's replicas of every S slice
    if ((rc = make_map_bf16(&g.tmS, g.S16, 2ull * bn, g.n_pad, pair ? bn / 2 : bn))) return rc;
  }
  // list scheduling of groups onto CTA slots
  std::vector<int> order(gl.size());
  for (size_t k = 0; k < order.size(); ++k) order[k] = static_cast<int>(k);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return gl[x].dur > gl[y].dur; });
  std::vector<double> free_at(capacity, 0.0);
  std::vector<std::vector<TcItem>> per_slot(capacity);
  std::vector<int> slots(capacity);
  for (int gi : order) {
    for (int s = 0; s < capacity; ++s) slots[s] = s;
    std::stable_sort(slots.begin(), slots.end(), [&](int x, int y) { return free_at[x] < free_at[y]; });
    const int nb = gl[gi].nb;
    double start = 0.0;
    for (int b = 0; b < nb; ++b) start = std::max(start, free_at[slots[b]]);
    for (int b = 0; b < nb; ++b) {
      if (!(withhold_tile && gi == 0 && b == nb - 1)) per_slot[slots[b]].push_back(TcItem{gi, b});
      free_at[slots[b]] = start + gl[gi].dur;
    }
  }
  int grid = 0;  // units launched (CTAs, or CTA pairs)
  for (int s = 0; s < capacity; ++s)
    if (!per_slot[s].empty()) grid = std::max(grid, s % ctas + 1);
  // the kernel's work lists in its order: pipeline-major, sub * grid + cta
  TcItem* hi = reinterpret_cast<TcItem*>(plan->host.data() + off_items);
  int32_t* hf = reinterpret_cast<int32_t*>(plan->host.data() + off_first);
  int32_t pos = 0;
  for (int p = 0; p < subs; ++p)
    for (int c = 0; c < grid; ++c) {
      hf[p * grid + c] = pos;
      for (const TcItem& it : per_slot[p * ctas + c]) hi[pos++] = it;
    }
  hf[subs * grid] = pos;
  plan->dev = base;
  plan->groups_off = 0;
  plan->items_off = off_items;
  plan->first_off = off_first;
  plan->flags_off = off_flags;
  plan->flags_bytes = off_state - off_flags;  // flags, done counters and 2H sums
  plan->grid = pair ? 2 * grid : grid;  // CTAs launched
  plan->bn = jobs[0].bn;
  plan->pair = pair;
  plan->f8 = f8;
  plan->status = status;
  plan->makespan = *std::max_element(free_at.begin(), free_at.end());
  return NMFA_OK;
}

void tc_plan_set_streams(TcPlan* plan, const uint32_t* stream_ids) {
  TcGroup* hg = reinterpret_cast<TcGroup*>(plan->host.data() + plan->groups_off);
  for (size_t k = 0; k < plan->group_job.size(); ++k) hg[k].stream = stream_ids[plan->group_job[k]];
}

// Upload the plan (group descriptors, items, per-pipeline offsets) from kernel
// parameters: no host-pinned buffer and no allocation, so it can be recorded in a
// CUDA graph.  Stream-ordered.
int tc_upload_plan(const TcPlan& plan, cudaStream_t st) {
  const size_t total = plan.flags_off;  // descriptors, items and offsets precede the flags
  TcUpload u;
  for (size_t off = 0; off < total; off += kUploadBytes) {
    const size_t chunk = std::min<size_t>(kUploadBytes, total - off);
    u.bytes = static_cast<uint32_t>(chunk);
    std::memcpy(u.data, plan.host.data() + off, chunk);
    tc_upload_kernel<<<1, 256, 0, st>>>(u, reinterpret_cast<uint4*>(static_cast<char*>(plan.dev) + off));
    count_launch();
    const int rc = cuda_error(cudaGetLastError(), "plan upload");
    if (rc) return rc;
  }
  return NMFA_OK;
}

// Enqueue: upload the plan if asked, clear the epoch counters, launch the
// persistent kernel.  Everything is stream-ordered and capturable.
int tc_enqueue_plan(const TcPlan& plan, bool upload, cudaStream_t st) {
  int rc;
  if (upload && (rc = tc_upload_plan(plan, st))) return rc;
  if ((rc = cuda_error(cudaMemsetAsync(static_cast<char*>(plan.dev) + plan.flags_off, 0, plan.flags_bytes, st),
                       "flag reset")))
    return rc;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(plan.grid, 1, 1);
  cfg.blockDim = dim3(plan.f8 ? (plan.bn == 256  ? TcShape<256, false, true>::kThreads
                                 : plan.bn == 64 ? TcShape<64, false, true>::kThreads
                                                 : TcShape<128, false, true>::kThreads)
                      : plan.pair      ? TcShape<128, true>::kThreads
                      : plan.bn == 64  ? TcShape<64>::kThreads
                      : plan.bn == 256 ? TcShape<256>::kThreads
                                       : TcShape<128>::kThreads,
                      1, 1);
  cfg.dynamicSmemBytes = plan.f8 ? (plan.bn == 256  ? TcShape<256, false, true>::kSmemBytes
                                     : plan.bn == 64 ? TcShape<64, false, true>::kSmemBytes
                                                     : TcShape<128, false, true>::kSmemBytes)
                         : plan.pair      ? TcShape<128, true>::kSmemBytes
                         : plan.bn == 64  ? TcShape<64>::kSmemBytes
                         : plan.bn == 256 ? TcShape<256>::kSmemBytes
                                          : TcShape<128>::kSmemBytes;
  cfg.stream = st;
  // cooperative: every CTA of the grid is resident at once (the tiles of a group wait
  // for one another); CTA pairs are clusters of two
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  attr[1].id = cudaLaunchAttributeClusterDimension;
  attr[1].val.clusterDim.x = 2;
  attr[1].val.clusterDim.y = 1;
  attr[1].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = plan.pair ? 2 : 1;
  const char* d = static_cast<const char*>(plan.dev);
  const TcGroup* dg = reinterpret_cast<const TcGroup*>(d + plan.groups_off);
  const TcItem* di = reinterpret_cast<const TcItem*>(d + plan.items_off);
  const int32_t* df = reinterpret_cast<const int32_t*>(d + plan.first_off);
  const cudaError_t ce = plan.f8 ? (plan.bn == 256  ? cudaLaunchKernelEx(&cfg, nmfa_tc_kernel<256, false, true>, dg, di, df,
                                                                       plan.status)
                                     : plan.bn == 64 ? cudaLaunchKernelEx(&cfg, nmfa_tc_kernel<64, false, true>, dg, di, df,
                                                                       plan.status)
                                                     : cudaLaunchKernelEx(&cfg, nmfa_tc_kernel<128, false, true>, dg, di, df,
                                                                       plan.status))
                         : plan.pair      ? cudaLaunchKernelEx(&cfg, nmfa_tc_kernel<128, true>, dg, di, df, plan.status)
                         : plan.bn == 64  ? cudaLaunchKernelEx(&cfg, nmfa_tc_kernel<64>, dg, di, df, plan.status)
                         : plan.bn == 256 ? cudaLaunchKernelEx(&cfg, nmfa_tc_kernel<256>, dg, di, df, plan.status)
                                          : cudaLaunchKernelEx(&cfg, nmfa_tc_kernel<128>, dg, di, df, plan.status);
  if ((rc = cuda_error(ce, "tensor kernel launch"))) return rc;
  count_launch();
  return NMFA_OK;
}

// FP8-stored couplings take the BF16 widths.  Their 64-replica tiles run one
// pipeline per CTA (the converter warps take the second pipeline's place), which
// fits: 64 is picked only where the tiles fill at most the SMs.  256-replica tiles
// convert each J slice once for twice the replicas but run on half the SMs, and
// measure slower wherever 128-replica tiles fit in one wave.  Results do not depend
// on the width.
int tc_pick_bn_for(const TcProblem& pb, int32_t replicas) { return tc_pick_bn(replicas, pb.n_pad); }

int tc_workspace_bytes(const TcProblem& pb, int32_t replicas, int64_t* bytes) {
  TcJob jb{};
  jb.pb = pb;
  jb.rp.replicas = replicas;
  jb.bn = tc_pick_bn_for(pb, replicas);
  return tc_plan_bytes(&jb, 1, bytes);
}

int launch_tc(const TcProblem& pb, const RunParams& rp, const TcWorkspace& ws, cudaStream_t st) {
  if (pb.n_pad % kBM != 0) return set_error(NMFA_EINVAL, "tensor path: n_pad must be a multiple of 128");
  TcJob jb{};
  jb.pb = pb;
  jb.rp = rp;
  jb.bn = tc_pick_bn_for(pb, rp.replicas);
  TcPlan plan;
  int rc = tc_build_plan(&jb, 1, ws.S16, ws.bytes, ws.status, &plan);
  if (rc) return rc;
  return tc_enqueue_plan(plan, true, st);
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
