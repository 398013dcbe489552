// engine_dev.h -- device data layout of the persistent batched engine (host + device).
//
// HBM layout (all allocated by the engine):
//   SlotDev[max_requests]     read-only request constants (decoded on the host)
//   SlotCtl[max_requests]     per-request work queue head, in-flight lane count, fair-share cap,
//                             state and the running sums of the completed id-block prefix
//   lane state, structure of arrays, one entry per lane (lanes = threads x T):
//       r (wrapped phase), v, hb (upper event bound), w (winding), c (64-bit Philox block
//       counter = Philox blocks of 4 steps consumed, a multiple of kBlockPhilox between kernel
//       blocks), gid (64-bit trajectory id), slot, budget
//   per request: IdBlockAcc[n_idblocks] + u32 histogram rows [rows][hist_bins], rows = n_idblocks
//       with a stop rule, ceil(n_traj / 2^31) without (+ optional int64 escape step per trajectory)
#pragma once

#include <cstdint>

#if defined(__CUDACC__)
#define FPT_HD __host__ __device__
#else
#define FPT_HD
#endif

namespace fpt {

enum : int { kSlotFree = 0, kSlotActive = 1, kSlotFinished = 2, kSlotCancelled = 3 };

// Code paths a warp can run: kind = model + 2 x integrator + 4 x ramp (underdamped / overdamped
// x Euler-Maruyama / Heun x constant / ramped bias).  A warp runs one kind at a time.
constexpr int kNumKinds = 8;

// Resident request slots an engine may have (the kernel keeps a per-slot view in shared memory).
constexpr int kMaxRequests = 1024;

// New trajectory ids a warp may hold beyond what its idle lanes need when it claims from a queue
// head (its reservoir, used by its next refills without an atomic).  Leftovers go back into the
// request's ring of suspended trajectories at the end of a launch, which therefore has room for
// kReserveIds per warp on top of twice the lanes.
constexpr int kReserveIds = 32;

// Philox blocks (of 4 steps) between re-bases of a trajectory's single-precision bias: gamma_k is
// formed as gs + nu dt (s + 1) with gs = gb + nu dt Jf and gb = gamma0 + nu dt 4 c_base in FP64,
// c_base the trajectory's own block count rounded down to a multiple of kRebaseBlocks, so the
// rounding depends only on the trajectory's step count, never on scheduling.
constexpr unsigned kRebaseBlocks = 1u << 20;

// Trajectory ids per histogram row of a request without a stop rule (its 32-bit counts cannot
// overflow); with a stop rule there is one row per id block.
constexpr uint64_t kHistRowIds = 1ull << 31;

// A trajectory suspended by preemption: everything needed to continue it exactly.
struct ParkEntry {
    float r, v;
    int w;
    unsigned c_lo, c_hi, gid_lo, gid_hi, pad;
};

// Exact accumulators of one block of stop_block (<= 2^32) consecutive trajectory ids.  The sums
// of k (< 2^48) and k^2 (< 2^96) are kept as sums of their 32-bit limbs, each in 64 bits, so a
// trajectory adds to them with plain atomic additions whose result nobody waits for (no carry
// to propagate); the scan kernel combines the limbs into 128-bit sums:
//   sum k = s1[0] + 2^32 s1[1],   sum k^2 = s2[0] + 2^32 s2[1] + 2^64 s2[2].
struct IdBlockAcc {
    unsigned int done, escaped, under, over;
    unsigned long long s1[2];   // limbs of the sum of escape steps
    unsigned long long s2[3];   // limbs of the sum of squared escape steps
};

// Exact quotient n / d for 0 <= n < 2^40 (trajectory indices; n_traj <= 2^40) and a 32-bit
// divisor d >= 1 by one multiply: with l = ceil(log2 d) and m = ceil(2^(40 + l) / d) < 2^41 + 1,
// floor(n / d) = floor(n m / 2^(40 + l)) (Granlund & Montgomery, "Division by invariant integers
// using multiplication", 1994, Thm. 4.2 with N = 40: 2^(N+l) <= m d <= 2^(N+l) + 2^l).
inline void id_block_magic(uint32_t d, uint64_t &m, int32_t &s) {
    int l = 0;
    while ((1ull << l) < d) ++l;
    s = 40 + l;
    const unsigned __int128 p = static_cast<unsigned __int128>(1) << s;
    m = static_cast<uint64_t>((p + d - 1) / d);
}

FPT_HD inline uint64_t id_block_quot(uint64_t n, uint64_t m, int32_t s) {
#if defined(__CUDA_ARCH__)
    const uint64_t hi = __umul64hi(n, m);
#else
    const uint64_t hi = static_cast<uint64_t>((static_cast<unsigned __int128>(n) * m) >> 64);
#endif
    const uint64_t lo = n * m;
    return s >= 64 ? hi >> (s - 64) : (lo >> s) | (hi << (64 - s));   // 40 <= s <= 72
}

struct SlotDev {
    // single-precision step constants
    float dt, A, amp, bmc, nudt, v0, r0, eb0;
    int32_t w0, kind;         // kind = model + 2 x integrator + 4 x ramp
    uint32_t key0, key1;
    // trajectories and budget
    uint64_t traj_offset, n_traj, max_steps, nblocks;   // nblocks = ceil(max_steps / 4)
    double gamma0, nudt_d;                               // double bias ramp
    float gb0;                // bias base of a trajectory at block 0 (set_progress at c = 0)
    uint32_t budget0;         // its event countdown at block 0
    // observable and histogram: x = out_a + out_b k
    int32_t output, hist_bins;
    double out_a, out_b, hist_lo, hist_hi, hist_inv_w;
    // prefix stop rule
    double stop_rse;
    uint32_t stop_block, n_idblocks;
    uint64_t ib_magic;        // id block of index i = id_block_quot(i, ib_magic, ib_shift)
    int32_t ib_shift;
    IdBlockAcc *acc;
    unsigned int *hist;        // rows x hist_bins
    int32_t hist_per_block;    // 1: row = id block (stop rule), 0: row = id / kHistRowIds
    uint32_t hist_rows;
    long long *per_traj;
    ParkEntry *park;           // ring of suspended trajectories
    unsigned park_cap;
};

struct SlotCtl {
    unsigned long long head;   // next trajectory index to hand out (may run past n_traj)
    int inflight;              // lanes integrating a trajectory of this request
    int state;                 // kSlot*
    unsigned int prefix;       // id blocks folded into the running sums
    unsigned int reserved;
    unsigned long long n_done, n_esc, s1_lo, s1_hi, s2_lo, s2_hi, under, over;
    // suspended-trajectory ring: pushes at launch end, committed by the scan, popped by refill
    unsigned park_tail, park_head, park_commit;
    int park_avail;            // committed entries not yet taken
    int park_used;             // entries pushed and not yet taken (bounds the ring)
    int reserved2;
};

struct LaneSoA {
    float *r, *v, *hb;
    int *w, *slot;
    unsigned int *c_lo, *c_hi, *gid_lo, *gid_hi, *budget;
};

// Global counters; kCntCheck collects the violated bounds of a build with FPT_CHECK (bit per
// check, see engine_kernels.cu), 0 otherwise.
enum : int { kCntUseful = 0, kCntEscapes = 1, kCntCensored = 2, kCntCheck = 3, kCntCount = 4 };

struct EngineDev {
    SlotDev *slots;
    SlotCtl *ctl;
    const int *caps;        // [max_requests] fair-share lane caps
    int *preempt;           // [max_requests] lanes to suspend at the end of this launch
    int *vacate;            // [kNumKinds] whole warps of each kind to suspend at the end of this launch
    const int *strict;      // [1] 1: never exceed the caps (someone is starved)
    const int *claim_warps; // [1] warps of each CTA (counted from warp 0) that claim new work:
                            // when there is less work than lanes it is spread over every SM
    const int *chunk_now;   // [1] blocks per warp of this launch (<= chunk_blocks)
    const int *act_list;    // [kNumKinds][max_requests] claimable slots per kind
    const int *act_count;   // [kNumKinds]
    LaneSoA lanes;
    int *warp_kind;         // kind each warp currently integrates (-1 idle)
    unsigned int *warp_cursor;
    unsigned long long *counters;
    unsigned int chunk_blocks;   // blocks per warp of a full launch
    int max_requests;
    unsigned int n_lanes;   // threads x trajectories per thread (lane state entries)
};

}  // namespace fpt
