// engine.cpp -- host side of the persistent batched FPT engine and its C ABI.
//
// One engine iteration:
//   1. admission: queued requests take a free slot when their device memory fits the budget;
//      their decoded constants (the set-up of Alg. 1 / Alg. 3) are copied into the slot
//      table and their accumulators are zeroed;
//   2. the claimable-slot lists and fair-share caps are refreshed (pinned host -> device);
//   3. one resident-kernel launch advances every lane by up to chunk_steps steps;
//   4. the scan kernel folds completed id blocks and applies the stop rule;
//   5. the per-slot status and counters come back to pinned host memory.
// Steps 2-5 are one CUDA graph.  Slots are reused only after no lane holds a trajectory of the
// old request (its in-flight count has reached zero).
//
// Iterations are pipelined one deep: iteration i+1 is enqueued before the host waits for
// iteration i and processes its status, so the GPU never idles while the host does admission,
// list building and status processing.  Two sets of pinned buffers (lists uploaded, status
// downloaded) and two graphs alternate.  Decisions taken on the host (admission, fair-share caps,
// preemption) therefore see the status of two launches back; completion and the stop rule are
// taken on the device by the scan kernel, so results do not depend on the lag.  fpt_step,
// checkpoints and destruction drain the pipeline.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "engine_dev.h"
#include "internal.h"

namespace fpt {
cudaError_t launch_engine_chunk(const EngineDev &E, int T, unsigned grid, unsigned block,
                                cudaStream_t s);
cudaError_t launch_engine_scan(const EngineDev &E, cudaStream_t s);
cudaError_t engine_chunk_occupancy(int T, int block, int *blocks_per_sm);
}  // namespace fpt

using namespace fpt;
using Clock = std::chrono::steady_clock;

namespace {
// NVTX range around a scope (header-only NVTX: a no-op unless a profiler is attached), so a
// timeline shows the host side of each engine iteration: admission and lists, enqueue, waiting
// for a launch and processing its status.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
}  // namespace

namespace {

enum Phase { kPending, kRunning, kFinished, kCancelled };

struct Request {
    uint64_t id = 0;
    fpt_params params{};
    Decoded dec;
    uint64_t n_traj = 0, seed = 0;
    int slot = -1;
    Phase phase = kPending;
    bool released = false;
    IdBlockAcc *acc = nullptr;
    unsigned *hist = nullptr;
    long long *per_traj = nullptr;
    ParkEntry *park = nullptr;
    uint32_t park_cap = 0;
    size_t bytes = 0;
    uint32_t stop_block = 4096, n_idblocks = 0;
    unsigned prefix = 0;
    fpt_sums sums{};
    fpt_result result{};
    Clock::time_point t_submit;
    bool suspending = false;          // checkpoint requested: no new work, lanes park
    bool quiesced = false;            // no lane holds a trajectory; all suspended ones committed
    // Iterations whose status may describe this request: from the first one enqueued after its
    // admission (earlier ones show the slot's previous occupant), and for the quiesced test
    // from the first one built with the suspension in force.
    uint64_t admit_seq = 0, suspend_seq = UINT64_MAX;
    std::vector<uint8_t> restore;     // checkpoint payload to load at admission
};

// Serialised request (fpt_checkpoint / fpt_restore): header, then SlotCtl, id-block accumulators,
// histogram rows, per-trajectory steps (if kept) and suspended trajectories.
struct CkptHeader {
    uint64_t magic, version;
    fpt_params params;
    uint64_t n_traj, seed;
    uint32_t stop_block, n_idblocks;
    uint64_t n_park, has_per_traj;
};
constexpr uint64_t kCkptMagic = 0x5450464B43505446ull;   // "FTPCKFPT"
constexpr uint64_t kCkptVersion = 3;   // 3: id-block sums as 32-bit limbs, histogram rows per hist_rows

// Ring of suspended trajectories: twice the lanes (suspensions) plus every warp's reservoir of
// unstarted ids returned at a launch end, and never more than the request's trajectories.
uint32_t park_capacity(uint64_t n_traj, unsigned lanes) {
    const uint64_t warps = (lanes + 31) / 32;
    const uint64_t cap = std::min<uint64_t>(n_traj, 2ull * lanes + static_cast<uint64_t>(kReserveIds) * warps);
    return static_cast<uint32_t>(std::max<uint64_t>(cap, 1));
}

// Histogram rows of a request: one per id block when the prefix stop rule may cut the result
// (the result's histogram is the sum of the rows of its prefix), otherwise one per 2^31 ids
// (32-bit counts cannot overflow) -- a single row up to 2^31 trajectories.
uint64_t hist_rows(const fpt_params &p, uint64_t n_traj, uint32_t B) {
    if (p.stop_rse > 0.0) return (n_traj + B - 1) / B;
    return (n_traj + kHistRowIds - 1) / kHistRowIds;
}

size_t request_bytes(const fpt_params &p, uint64_t n_traj, uint32_t B, unsigned lanes) {
    const uint64_t nb = (n_traj + B - 1) / B;
    size_t bytes = nb * sizeof(IdBlockAcc) + hist_rows(p, n_traj, B) * static_cast<size_t>(p.hist_bins) * 4;
    bytes += static_cast<size_t>(park_capacity(n_traj, lanes)) * sizeof(ParkEntry);
    if (p.keep_per_traj) bytes += n_traj * 8;
    return bytes;
}

}  // namespace

// Host side of one in-flight iteration: the lists it uploads, the status it downloads, its
// events and its graph.  Two alternate.
struct IterIO {
    int *caps = nullptr, *act = nullptr, *act_count = nullptr;
    int *preempt = nullptr, *flags = nullptr;   // flags: vacate[kNumKinds], strict, claim_warps,
                                                // blocks per warp of the launch
    SlotCtl *ctl = nullptr;                     // status download target
    unsigned long long *counters = nullptr;     // counters download target
    cudaEvent_t k0 = nullptr, k1 = nullptr;     // around the resident kernel
    cudaEvent_t done = nullptr;                 // after the downloads
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t seq = 0;                           // number of the iteration that used these buffers
    unsigned chunk_blocks = 0;                  // blocks per warp of that launch
};

// Flags uploaded with each launch: vacate[kNumKinds], strict, claim_warps, blocks per warp.
constexpr int kNumFlags = kNumKinds + 3;

// Launches after its admission during which a request that fits in the lanes counts as young
// (the launch length is then the engine's young_chunk_steps).
constexpr uint64_t kYoungLaunches = 16;

struct fpt_engine {
    fpt_engine_config cfg{};
    int device = 0;
    cudaStream_t stream = nullptr, io = nullptr;
    bool own_stream = false;
    int sms = 0, grid = 0, block = 256, T = 2, maxr = 256;
    unsigned lanes = 0, chunk_blocks = 0;
    unsigned young_blocks = 0;    // blocks per warp of a launch while a small request is young
    uint64_t lane_slots = 0;      // lanes x steps offered by the processed launches
    // device
    SlotDev *d_slots = nullptr;
    SlotCtl *d_ctl = nullptr;
    int *d_caps = nullptr, *d_act = nullptr, *d_act_count = nullptr;
    int *d_preempt = nullptr, *d_vacate = nullptr, *d_strict = nullptr;
    void *d_lane_mem = nullptr;
    int *d_warp_kind = nullptr;
    unsigned *d_warp_cursor = nullptr;
    unsigned long long *d_counters = nullptr;
    EngineDev dev{};
    // pinned host: admission staging, the last processed status and counters (stable copies read
    // by fpt_poll, admission and list building), and the two alternating iteration buffers
    SlotDev *h_slots = nullptr;
    SlotCtl *h_ctl = nullptr, *h_ctl_init = nullptr;
    unsigned long long *h_counters = nullptr;
    uint64_t preempted = 0;
    IterIO iters[2];
    int next_io = 0;              // buffers of the next iteration to enqueue
    uint64_t enq_seq = 0;         // number of the next iteration to enqueue
    uint64_t status_seq = UINT64_MAX;   // number of the iteration h_ctl comes from (none yet)
    int flight[2] = {0, 0};       // enqueued, unprocessed iterations (buffer index), oldest first
    std::atomic<int> n_flight{0};   // changed by the driving thread, read by the service loop
    double kernel_ms = 0.0;       // summed resident-kernel time (events inside each iteration)
    bool capturing = false;
    // bookkeeping
    std::mutex mu, drive_mu;
    std::condition_variable cv_work, cv_done;
    std::thread service;
    bool stop = false;
    std::deque<uint64_t> pending;
    std::map<uint64_t, std::unique_ptr<Request>> reqs;
    std::vector<uint64_t> slot_req;
    uint64_t next_id = 1;
    uint64_t budget = 0, mem_used = 0;
    uint64_t iterations = 0;
    bool broken = false;
    std::string error;
};

namespace {

thread_local std::string t_engine_error;

fpt_status fail(fpt_engine *e, fpt_status st, const std::string &m) {
    if (e) {
        e->error = m;
        t_engine_error = m;
    } else {
        set_error(m);
    }
    return st;
}

#define CK(call)                                                                         \
    do {                                                                                 \
        cudaError_t _e = (call);                                                         \
        if (_e != cudaSuccess) {                                                         \
            e->broken = true;                                                            \
            return fail(e, FPT_ECUDA, std::string(#call) + ": " + cudaGetErrorString(_e)); \
        }                                                                                \
    } while (0)

void free_request_buffers(Request &R, fpt_engine *e) {
    if (R.acc) cudaFree(R.acc);
    if (R.hist) cudaFree(R.hist);
    if (R.per_traj) cudaFree(R.per_traj);
    if (R.park) cudaFree(R.park);
    R.acc = nullptr;
    R.hist = nullptr;
    R.per_traj = nullptr;
    R.park = nullptr;
    e->mem_used -= R.bytes;
    R.bytes = 0;
}

// Admit queued requests (called with mu held, on the driving thread).
fpt_status admit(fpt_engine *e) {
    for (auto it = e->pending.begin(); it != e->pending.end();) {
        Request &R = *e->reqs[*it];
        if (R.released) {
            it = e->pending.erase(it);
            e->reqs.erase(R.id);
            continue;
        }
        int s = -1;
        for (int i = 0; i < e->maxr; ++i)
            if (e->slot_req[i] == 0) {
                s = i;
                break;
            }
        if (s < 0) break;
        const size_t bytes = request_bytes(R.params, R.n_traj, R.stop_block, e->lanes);
        if (e->mem_used + bytes > e->budget) {
            ++it;
            continue;
        }
        const uint64_t nb = R.n_idblocks;
        CK(cudaMalloc(&R.acc, nb * sizeof(IdBlockAcc)));
        const size_t hist_bytes = hist_rows(R.params, R.n_traj, R.stop_block) * static_cast<size_t>(R.params.hist_bins) * 4;
        CK(cudaMalloc(&R.hist, hist_bytes));
        CK(cudaMemsetAsync(R.acc, 0, nb * sizeof(IdBlockAcc), e->stream));
        CK(cudaMemsetAsync(R.hist, 0, hist_bytes, e->stream));
        if (R.params.keep_per_traj) {
            CK(cudaMalloc(&R.per_traj, R.n_traj * 8));
            CK(cudaMemsetAsync(R.per_traj, 0xFF, R.n_traj * 8, e->stream));
        }
        R.park_cap = park_capacity(R.n_traj, e->lanes);
        CK(cudaMalloc(&R.park, static_cast<size_t>(R.park_cap) * sizeof(ParkEntry)));
        R.bytes = bytes;
        e->mem_used += bytes;
        const Decoded &d = R.dec;
        SlotDev &S = e->h_slots[s];
        std::memset(&S, 0, sizeof(S));
        S.dt = d.dt_f;
        S.A = d.A_f;
        S.amp = d.amp_f;
        S.bmc = d.bmc_f;
        S.nudt = d.nudt_f;
        S.v0 = d.v0_f;
        S.r0 = d.r0_f;
        S.eb0 = d.eb0_f;
        S.w0 = d.w0;
        S.kind = d.kind;
        S.key0 = static_cast<uint32_t>(R.seed);
        S.key1 = static_cast<uint32_t>(R.seed >> 32);
        S.traj_offset = R.params.traj_offset;
        S.n_traj = R.n_traj;
        S.max_steps = d.max_steps;
        S.nblocks = (d.max_steps + 3) / 4;
        S.gamma0 = d.gamma0;
        S.nudt_d = d.nudt;
        // the bias base and event countdown of a trajectory at block 0, as the kernel's
        // set_progress forms them (c = c_base = 0; the re-base and carry counts are whole)
        S.gb0 = static_cast<float>(d.gamma0 + d.nudt * static_cast<double>(0ull));
        {
            const uint64_t to_end = S.nblocks, to_base = kRebaseBlocks, to_carry = 0x100000000ull;
            uint64_t m = to_end < to_base ? to_end : to_base;
            m = m < to_carry ? m : to_carry;
            S.budget0 = static_cast<uint32_t>((m + kBlockPhilox - 1) / kBlockPhilox);
        }
        S.output = d.output;
        S.hist_bins = d.hist_bins;
        S.out_a = d.out_a;
        S.out_b = d.out_b;
        S.hist_lo = d.hist_lo;
        S.hist_hi = d.hist_hi;
        S.hist_inv_w = d.hist_inv_w;
        S.stop_rse = R.params.stop_rse;
        S.stop_block = R.stop_block;
        S.n_idblocks = R.n_idblocks;
        id_block_magic(R.stop_block, S.ib_magic, S.ib_shift);
        S.acc = R.acc;
        S.hist = R.hist;
        S.hist_per_block = R.params.stop_rse > 0.0 ? 1 : 0;
        S.hist_rows = static_cast<uint32_t>(hist_rows(R.params, R.n_traj, R.stop_block));
        S.per_traj = R.per_traj;
        S.park = R.park;
        S.park_cap = R.park_cap;
        CK(cudaMemcpyAsync(e->d_slots + s, &S, sizeof(SlotDev), cudaMemcpyHostToDevice, e->stream));
        SlotCtl &C = e->h_ctl_init[s];
        std::memset(&C, 0, sizeof(C));
        if (!R.restore.empty()) {
            // continue a checkpointed request: counters, accumulators, histogram rows,
            // per-trajectory steps and suspended trajectories (re-based to ring index 0)
            const uint8_t *q = R.restore.data();
            const CkptHeader &H = *reinterpret_cast<const CkptHeader *>(q);
            q += sizeof(CkptHeader);
            std::memcpy(&C, q, sizeof(SlotCtl));
            q += sizeof(SlotCtl);
            const size_t acc_b = nb * sizeof(IdBlockAcc), hist_b = hist_bytes;
            CK(cudaMemcpyAsync(R.acc, q, acc_b, cudaMemcpyHostToDevice, e->stream));
            q += acc_b;
            CK(cudaMemcpyAsync(R.hist, q, hist_b, cudaMemcpyHostToDevice, e->stream));
            q += hist_b;
            if (H.has_per_traj) {
                if (R.per_traj)
                    CK(cudaMemcpyAsync(R.per_traj, q, R.n_traj * 8, cudaMemcpyHostToDevice, e->stream));
                q += R.n_traj * 8;
            }
            const unsigned np = static_cast<unsigned>(H.n_park);
            if (np) CK(cudaMemcpyAsync(R.park, q, np * sizeof(ParkEntry), cudaMemcpyHostToDevice, e->stream));
            C.inflight = 0;
            C.park_head = 0;
            C.park_tail = C.park_commit = np;
            C.park_avail = C.park_used = static_cast<int>(np);
            CK(cudaStreamSynchronize(e->stream));   // the payload is host memory we free below
            R.restore.clear();
            R.restore.shrink_to_fit();
        }
        C.state = kSlotActive;
        CK(cudaMemcpyAsync(e->d_ctl + s, &C, sizeof(SlotCtl), cudaMemcpyHostToDevice, e->stream));
        e->slot_req[s] = R.id;
        R.slot = s;
        R.phase = kRunning;
        R.admit_seq = e->enq_seq;   // the coming launch is the first to see it
        it = e->pending.erase(it);
    }
    return FPT_OK;
}

// Claimable lists, fair-share caps and preemption orders for the next launch (mu held).
// Fair share = lanes / running requests.  A request is starved when it has work (unclaimed
// ids or suspended trajectories) and holds less than half of min(share, its demand).  While
// anyone is starved: caps are strict, requests above their share suspend the excess lanes at
// the end of the launch, and if a starved request's kind (model x integrator) differs, whole
// warps of other kinds vacate so they can switch.
// Whether the last processed status describes request R (and not its slot's previous occupant).
bool fresh(const fpt_engine *e, const Request &R) {
    return e->status_seq != UINT64_MAX && e->status_seq >= R.admit_seq;
}

void build_lists(fpt_engine *e, IterIO &B) {
    int cnt[kNumKinds] = {};
    int active = 0;
    for (int s = 0; s < e->maxr; ++s) {
        B.preempt[s] = 0;
        if (!e->slot_req[s]) continue;
        Request &R = *e->reqs[e->slot_req[s]];
        if (R.phase != kRunning) continue;
        if (R.suspending) {                 // checkpoint: no new work, every lane suspends
            B.preempt[s] = 1 << 30;
            if (R.suspend_seq == UINT64_MAX) R.suspend_seq = e->enq_seq;
            continue;
        }
        B.act[R.dec.kind * e->maxr + cnt[R.dec.kind]++] = s;
        ++active;
    }
    for (int k = 0; k < kNumKinds; ++k) B.act_count[k] = cnt[k];
    const int share = active ? static_cast<int>((e->lanes + active - 1) / active) : 0;
    const int cap = active ? share + 32 : 0;
    for (int s = 0; s < e->maxr; ++s) B.caps[s] = cap;
    for (int k = 0; k <= kNumKinds; ++k) B.flags[k] = 0;
    for (int s = 0; s < e->maxr; ++s)
        if (B.preempt[s]) B.flags[kNumKinds] = 1;   // keep a suspending request's lanes from refilling
    // With fewer trajectories in flight and queued than lanes, only the first warps of every CTA
    // claim new work, so the busy warps spread over all SMs instead of filling a few of them.
    {
        int64_t work = 0;
        for (int s = 0; s < e->maxr; ++s) {
            if (!e->slot_req[s]) continue;
            const Request &R = *e->reqs[e->slot_req[s]];
            if (R.phase != kRunning || R.suspending) continue;
            const SlotCtl &C = e->h_ctl[s];
            if (fresh(e, R) && C.state == kSlotActive) {
                const uint64_t head = std::min<uint64_t>(C.head, R.n_traj);
                work += static_cast<int64_t>(R.n_traj - head) + std::max(C.inflight, 0) +
                        std::max(C.park_avail, 0);
            } else {
                work += static_cast<int64_t>(R.n_traj);   // admitted for the coming launch
            }
        }
        const int64_t per_warp = 32ll * e->T * e->grid;
        const int64_t warps = (work + per_warp - 1) / per_warp;
        B.flags[kNumKinds + 1] =
            static_cast<int>(std::min<int64_t>(std::max<int64_t>(warps, 1), e->block / 32));
    }
    // Launch length: short while a request that fits in the lanes is young, so it waits fewer
    // steps of the others for its admission, its lanes and the status that reports its result.
    B.chunk_blocks = e->chunk_blocks;
    if (e->young_blocks)
        for (int s = 0; s < e->maxr; ++s) {
            if (!e->slot_req[s]) continue;
            const Request &R = *e->reqs[e->slot_req[s]];
            if (R.phase == kRunning && !R.suspending && R.n_traj <= e->lanes &&
                e->enq_seq < R.admit_seq + kYoungLaunches) {
                B.chunk_blocks = e->young_blocks;
                break;
            }
        }
    B.flags[kNumKinds + 2] = static_cast<int>(B.chunk_blocks);
    if (active < 2) return;
    int64_t deficit[kNumKinds] = {};
    bool over[kNumKinds] = {};
    for (int s = 0; s < e->maxr; ++s) {
        if (!e->slot_req[s]) continue;
        Request &R = *e->reqs[e->slot_req[s]];
        if (R.phase != kRunning || R.suspending) continue;
        const SlotCtl &C = e->h_ctl[s];
        // A request without a status yet was just admitted: it holds no lane, so it is starved
        // from its first launch on and the requests above their share suspend lanes for it at
        // the end of that launch (waiting for its first status would cost two launches).
        const bool known = fresh(e, R);
        if (known && C.state != kSlotActive) continue;     // finishing
        int64_t inflight = 0, remaining = static_cast<int64_t>(R.n_traj);
        if (known) {
            const int64_t unclaimed = C.head < R.n_traj ? static_cast<int64_t>(R.n_traj - C.head) : 0;
            inflight = C.inflight;
            remaining = unclaimed + std::max(C.park_avail, 0);
        }
        const int64_t want = std::min<int64_t>(share, inflight + remaining);
        if (remaining > 0 && inflight < want / 2) deficit[R.dec.kind] += want - inflight;
        if (known && C.inflight > share) over[R.dec.kind] = true;
    }
    int64_t total_deficit = 0;
    for (int k = 0; k < kNumKinds; ++k) total_deficit += deficit[k];
    if (total_deficit == 0) return;
    B.flags[kNumKinds] = 1;   // strict caps
    for (int s = 0; s < e->maxr; ++s) {
        if (!e->slot_req[s]) continue;
        Request &R = *e->reqs[e->slot_req[s]];
        if (R.phase != kRunning || R.suspending) continue;
        const SlotCtl &C = e->h_ctl[s];
        if (!fresh(e, R) || C.state != kSlotActive || C.inflight <= share) continue;
        const int room = static_cast<int>(R.park_cap) - std::max(C.park_used, 0);
        B.preempt[s] = std::max(0, std::min(C.inflight - share, room));
        e->preempted += static_cast<uint64_t>(B.preempt[s]);
    }
    const int64_t lanes_per_warp = 32ll * e->T;
    for (int m = 0; m < kNumKinds; ++m) {
        const int64_t others = total_deficit - deficit[m];
        if (others > 0 && over[m])
            B.flags[m] = static_cast<int>((others + lanes_per_warp - 1) / lanes_per_warp);
    }
}

fpt_status enqueue_iteration(fpt_engine *e, IterIO &B) {
    if (B.exec) {
        CK(cudaGraphLaunch(B.exec, e->stream));
        return FPT_OK;
    }
    CK(cudaMemcpyAsync(e->d_caps, B.caps, e->maxr * sizeof(int), cudaMemcpyHostToDevice, e->stream));
    CK(cudaMemcpyAsync(e->d_preempt, B.preempt, e->maxr * sizeof(int), cudaMemcpyHostToDevice, e->stream));
    CK(cudaMemcpyAsync(e->d_vacate, B.flags, kNumFlags * sizeof(int), cudaMemcpyHostToDevice,
                       e->stream));
    CK(cudaMemcpyAsync(e->d_act, B.act, kNumKinds * e->maxr * sizeof(int), cudaMemcpyHostToDevice,
                       e->stream));
    CK(cudaMemcpyAsync(e->d_act_count, B.act_count, kNumKinds * sizeof(int), cudaMemcpyHostToDevice,
                       e->stream));
    const unsigned evflags = e->capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
    CK(cudaEventRecordWithFlags(B.k0, e->stream, evflags));
    CK(launch_engine_chunk(e->dev, e->T, e->grid, e->block, e->stream));
    CK(cudaEventRecordWithFlags(B.k1, e->stream, evflags));
    CK(launch_engine_scan(e->dev, e->stream));
    CK(cudaMemcpyAsync(B.ctl, e->d_ctl, e->maxr * sizeof(SlotCtl), cudaMemcpyDeviceToHost, e->stream));
    CK(cudaMemcpyAsync(B.counters, e->d_counters, kCntCount * sizeof(unsigned long long),
                       cudaMemcpyDeviceToHost, e->stream));
    return FPT_OK;
}

void finalize(fpt_engine *e, Request &R, const SlotCtl &C) {
    R.prefix = C.prefix;
    R.sums.n_done = C.n_done;
    R.sums.n_escaped = C.n_esc;
    R.sums.s1_lo = C.s1_lo;
    R.sums.s1_hi = C.s1_hi;
    R.sums.s2_lo = C.s2_lo;
    R.sums.s2_hi = C.s2_hi;
    R.sums.under = C.under;
    R.sums.over = C.over;
    std::memset(&R.result, 0, sizeof(R.result));
    R.result.state = FPT_OK;
    R.result.n_used = C.n_done;
    sums_to_result(R.dec, R.sums, &R.result);
    const unsigned __int128 s1 = (static_cast<unsigned __int128>(C.s1_hi) << 64) | C.s1_lo;
    const unsigned __int128 tot =
        s1 + static_cast<unsigned __int128>(C.n_done - C.n_esc) * R.dec.max_steps;
    R.result.steps_total = (tot >> 64) ? UINT64_MAX : static_cast<uint64_t>(tot);
    R.result.latency_s = std::chrono::duration<double>(Clock::now() - R.t_submit).count();
    (void)e;
}

// Read the status of the last processed iteration (mu held).
void process_status(fpt_engine *e) {
    for (int s = 0; s < e->maxr; ++s) {
        if (!e->slot_req[s]) continue;
        Request &R = *e->reqs[e->slot_req[s]];
        if (!fresh(e, R)) continue;   // launched before R was admitted: the previous occupant
        const SlotCtl &C = e->h_ctl[s];
        if (R.phase == kRunning && C.state == kSlotFinished) {
            finalize(e, R, C);
            R.phase = kFinished;
        }
        if (R.phase == kRunning && R.suspending && R.suspend_seq != UINT64_MAX &&
            e->status_seq >= R.suspend_seq && C.inflight == 0 && C.park_commit == C.park_tail)
            R.quiesced = true;
        if ((R.phase == kFinished || R.phase == kCancelled) && C.state != kSlotActive &&
            C.inflight == 0) {
            e->slot_req[s] = 0;
            R.slot = -1;
            if (R.released) {
                free_request_buffers(R, e);
                e->reqs.erase(R.id);
            }
        }
    }
}

// Wait for the oldest enqueued iteration and take its status: stable copies for fpt_poll,
// admission and list building, finished requests, freed slots, counters and kernel time.
fpt_status complete_oldest(fpt_engine *e) {
    NvtxRange range("fpt: wait and process status");
    IterIO &B = e->iters[e->flight[0]];
    CK(cudaEventSynchronize(B.done));
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, B.k0, B.k1));
    {
        std::lock_guard<std::mutex> lk(e->mu);
        std::memcpy(e->h_ctl, B.ctl, e->maxr * sizeof(SlotCtl));
        std::memcpy(e->h_counters, B.counters, kCntCount * sizeof(unsigned long long));
        e->status_seq = B.seq;
        process_status(e);
        ++e->iterations;
        e->lane_slots += static_cast<uint64_t>(e->lanes) * B.chunk_blocks * kBlockSteps;
        e->kernel_ms += ms;
    }
    e->flight[0] = e->flight[1];
    --e->n_flight;
    e->cv_done.notify_all();
    return FPT_OK;
}

// One engine iteration: admission and lists from the last processed status, enqueue, then
// process the previous iteration's status while this one runs (at most one iteration stays
// enqueued and unprocessed when this returns).
fpt_status iteration(fpt_engine *e) {
    if (e->broken) return fail(e, FPT_ECUDA, "engine is in an error state: " + e->error);
    if (e->n_flight == 2) {
        const fpt_status st = complete_oldest(e);
        if (st != FPT_OK) return st;
    }
    IterIO &B = e->iters[e->next_io];
    {
        NvtxRange range("fpt: admission and lists");
        std::lock_guard<std::mutex> lk(e->mu);
        fpt_status st = admit(e);
        if (st != FPT_OK) return st;
        build_lists(e, B);
    }
    B.seq = e->enq_seq++;
    NvtxRange range("fpt: enqueue iteration");
    fpt_status st = enqueue_iteration(e, B);
    if (st != FPT_OK) return st;
    CK(cudaEventRecord(B.done, e->stream));
    e->flight[e->n_flight.load()] = e->next_io;
    ++e->n_flight;
    e->next_io ^= 1;
    if (e->n_flight == 2) return complete_oldest(e);
    return FPT_OK;
}

// Process every enqueued iteration (the device has finished all of them on return).
fpt_status drain(fpt_engine *e) {
    while (e->n_flight > 0) {
        const fpt_status st = complete_oldest(e);
        if (st != FPT_OK) return st;
    }
    return FPT_OK;
}

bool has_work(fpt_engine *e) {
    if (!e->pending.empty()) return true;
    for (int s = 0; s < e->maxr; ++s)
        if (e->slot_req[s]) return true;
    return false;
}

void service_loop(fpt_engine *e) {
    for (;;) {
        bool work;
        {
            std::unique_lock<std::mutex> lk(e->mu);
            e->cv_work.wait(lk, [&] { return e->stop || has_work(e) || e->n_flight > 0; });
            if (e->stop) return;
            work = has_work(e);
        }
        std::lock_guard<std::mutex> dk(e->drive_mu);
        if ((work ? iteration(e) : drain(e)) != FPT_OK) {
            e->cv_done.notify_all();
            return;
        }
    }
}

fpt_status capture_graph(fpt_engine *e, IterIO &B) {
    CK(cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal));
    fpt_status st = FPT_OK;
    {
        B.exec = nullptr;
        e->capturing = true;
        st = enqueue_iteration(e, B);
        e->capturing = false;
    }
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(e->stream, &g);
    if (st != FPT_OK) return st;
    CK(ce);
    B.graph = g;
    CK(cudaGraphInstantiate(&B.exec, B.graph, 0));
    return FPT_OK;
}

void destroy_all(fpt_engine *e) {
    if (e->service.joinable()) {
        {
            std::lock_guard<std::mutex> lk(e->mu);
            e->stop = true;
        }
        e->cv_work.notify_all();
        e->service.join();
    }
    cudaSetDevice(e->device);
    if (e->stream) cudaStreamSynchronize(e->stream);
    e->n_flight = 0;
    for (auto &kv : e->reqs) free_request_buffers(*kv.second, e);
    e->reqs.clear();
    for (IterIO &B : e->iters) {
        if (B.exec) cudaGraphExecDestroy(B.exec);
        if (B.graph) cudaGraphDestroy(B.graph);
        cudaFreeHost(B.caps);
        cudaFreeHost(B.act);
        cudaFreeHost(B.act_count);
        cudaFreeHost(B.preempt);
        cudaFreeHost(B.flags);
        cudaFreeHost(B.ctl);
        cudaFreeHost(B.counters);
        if (B.k0) cudaEventDestroy(B.k0);
        if (B.k1) cudaEventDestroy(B.k1);
        if (B.done) cudaEventDestroy(B.done);
    }
    cudaFree(e->d_slots);
    cudaFree(e->d_ctl);
    cudaFree(e->d_caps);
    cudaFree(e->d_act);
    cudaFree(e->d_act_count);
    cudaFree(e->d_preempt);
    cudaFree(e->d_vacate);
    cudaFree(e->d_lane_mem);
    cudaFree(e->d_warp_kind);
    cudaFree(e->d_warp_cursor);
    cudaFree(e->d_counters);
    cudaFreeHost(e->h_slots);
    cudaFreeHost(e->h_ctl);
    cudaFreeHost(e->h_ctl_init);
    cudaFreeHost(e->h_counters);
    if (e->io) cudaStreamDestroy(e->io);
    if (e->own_stream && e->stream) cudaStreamDestroy(e->stream);
}

fpt_status create_impl(const fpt_engine_config *cfg_in, fpt_engine *e) {
    fpt_engine_config cfg{};
    if (cfg_in) cfg = *cfg_in;
    else cfg.use_graph = 1;
    e->cfg = cfg;
    e->device = cfg.device;
    int ndev = 0;
    CK(cudaGetDeviceCount(&ndev));
    if (cfg.device < 0 || cfg.device >= ndev) return fail(e, FPT_EINVAL, "bad device ordinal");
    CK(cudaSetDevice(cfg.device));
    e->maxr = cfg.max_requests > 0 ? cfg.max_requests : 256;
    if (e->maxr > kMaxRequests) return fail(e, FPT_EINVAL, "max_requests must be <= 1024");
    e->T = cfg.traj_per_thread > 0 ? cfg.traj_per_thread : 1;
    if (e->T != 1 && e->T != 2) return fail(e, FPT_EINVAL, "traj_per_thread must be 1 or 2");
    const int max_block = e->T == 1 ? 640 : 256;
    e->block = cfg.threads_per_block > 0 ? cfg.threads_per_block : max_block;
    if (e->block % 32 || e->block > max_block)
        return fail(e, FPT_EINVAL, "threads_per_block: multiple of 32, <= 640 (one trajectory per "
                                   "thread) or <= 256 (two)");
    const uint32_t chunk = cfg.chunk_steps ? cfg.chunk_steps : 16384;
    if (chunk % kBlockSteps || chunk > (1u << 24))
        return fail(e, FPT_EINVAL, "chunk_steps: multiple of 16 (the kernel's block), <= 2^24");
    e->chunk_blocks = chunk / kBlockSteps;
    if (cfg.young_chunk_steps % kBlockSteps || cfg.young_chunk_steps > chunk)
        return fail(e, FPT_EINVAL, "young_chunk_steps: multiple of 16, <= chunk_steps");
    e->young_blocks = cfg.young_chunk_steps / kBlockSteps;
    if (e->young_blocks == e->chunk_blocks) e->young_blocks = 0;
    CK(cudaDeviceGetAttribute(&e->sms, cudaDevAttrMultiProcessorCount, cfg.device));
    int bps = 0;
    CK(engine_chunk_occupancy(e->T, e->block, &bps));
    if (bps < 1) return fail(e, FPT_ECUDA, "resident kernel does not fit on an SM");
    if (cfg.blocks_per_sm > 0) bps = std::min(bps, cfg.blocks_per_sm);
    e->grid = e->sms * bps;
    e->lanes = static_cast<unsigned>(e->grid) * e->block * e->T;
    size_t free_b = 0, total_b = 0;
    CK(cudaMemGetInfo(&free_b, &total_b));
    e->budget = cfg.mem_budget_bytes ? cfg.mem_budget_bytes : free_b / 4;
    if (cfg.stream) {
        e->stream = static_cast<cudaStream_t>(cfg.stream);
    } else {
        CK(cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking));
        e->own_stream = true;
    }
    CK(cudaStreamCreateWithFlags(&e->io, cudaStreamNonBlocking));
    const int R = e->maxr;
    CK(cudaMalloc(&e->d_slots, R * sizeof(SlotDev)));
    CK(cudaMalloc(&e->d_ctl, R * sizeof(SlotCtl)));
    CK(cudaMalloc(&e->d_caps, R * sizeof(int)));
    CK(cudaMalloc(&e->d_act, kNumKinds * R * sizeof(int)));
    CK(cudaMalloc(&e->d_act_count, kNumKinds * sizeof(int)));
    CK(cudaMalloc(&e->d_preempt, R * sizeof(int)));
    CK(cudaMalloc(&e->d_vacate, kNumFlags * sizeof(int)));   // vacate[kNumKinds], strict, claim, chunk
    CK(cudaMemsetAsync(e->d_preempt, 0, R * sizeof(int), e->stream));
    CK(cudaMemsetAsync(e->d_vacate, 0, kNumFlags * sizeof(int), e->stream));
    const size_t L = e->lanes;
    CK(cudaMalloc(&e->d_lane_mem, L * 4 * 10));
    const unsigned nwarps = static_cast<unsigned>(e->grid) * e->block / 32;
    CK(cudaMalloc(&e->d_warp_kind, nwarps * sizeof(int)));
    CK(cudaMalloc(&e->d_warp_cursor, nwarps * sizeof(unsigned)));
    CK(cudaMalloc(&e->d_counters, kCntCount * sizeof(unsigned long long)));
    CK(cudaMemsetAsync(e->d_ctl, 0, R * sizeof(SlotCtl), e->stream));
    CK(cudaMemsetAsync(e->d_lane_mem, 0, L * 4 * 10, e->stream));
    char *m = static_cast<char *>(e->d_lane_mem);
    LaneSoA &ls = e->dev.lanes;
    ls.r = reinterpret_cast<float *>(m + 0 * L * 4);
    ls.v = reinterpret_cast<float *>(m + 1 * L * 4);
    ls.hb = reinterpret_cast<float *>(m + 2 * L * 4);
    ls.w = reinterpret_cast<int *>(m + 3 * L * 4);
    ls.slot = reinterpret_cast<int *>(m + 4 * L * 4);
    ls.c_lo = reinterpret_cast<unsigned *>(m + 5 * L * 4);
    ls.c_hi = reinterpret_cast<unsigned *>(m + 6 * L * 4);
    ls.gid_lo = reinterpret_cast<unsigned *>(m + 7 * L * 4);
    ls.gid_hi = reinterpret_cast<unsigned *>(m + 8 * L * 4);
    ls.budget = reinterpret_cast<unsigned *>(m + 9 * L * 4);
    CK(cudaMemsetAsync(ls.slot, 0xFF, L * 4, e->stream));
    CK(cudaMemsetAsync(e->d_warp_kind, 0xFF, nwarps * sizeof(int), e->stream));
    {   // stagger the warps' round-robin cursors so the first claims spread over all requests
        std::vector<unsigned> cur(nwarps);
        for (unsigned w = 0; w < nwarps; ++w) cur[w] = w;
        CK(cudaMemcpy(e->d_warp_cursor, cur.data(), nwarps * sizeof(unsigned),
                      cudaMemcpyHostToDevice));
    }
    CK(cudaMemsetAsync(e->d_counters, 0, kCntCount * sizeof(unsigned long long), e->stream));
    CK(cudaMallocHost(&e->h_slots, R * sizeof(SlotDev)));
    CK(cudaMallocHost(&e->h_ctl, R * sizeof(SlotCtl)));
    CK(cudaMallocHost(&e->h_ctl_init, R * sizeof(SlotCtl)));
    CK(cudaMallocHost(&e->h_counters, kCntCount * sizeof(unsigned long long)));
    std::memset(e->h_ctl, 0, R * sizeof(SlotCtl));
    std::memset(e->h_counters, 0, kCntCount * sizeof(unsigned long long));
    for (IterIO &B : e->iters) {
        CK(cudaMallocHost(&B.caps, R * sizeof(int)));
        CK(cudaMallocHost(&B.act, kNumKinds * R * sizeof(int)));
        CK(cudaMallocHost(&B.act_count, kNumKinds * sizeof(int)));
        CK(cudaMallocHost(&B.preempt, R * sizeof(int)));
        CK(cudaMallocHost(&B.flags, kNumFlags * sizeof(int)));
        CK(cudaMallocHost(&B.ctl, R * sizeof(SlotCtl)));
        CK(cudaMallocHost(&B.counters, kCntCount * sizeof(unsigned long long)));
        std::memset(B.caps, 0, R * sizeof(int));
        std::memset(B.act, 0, kNumKinds * R * sizeof(int));
        std::memset(B.act_count, 0, kNumKinds * sizeof(int));
        std::memset(B.preempt, 0, R * sizeof(int));
        std::memset(B.flags, 0, kNumFlags * sizeof(int));
        std::memset(B.ctl, 0, R * sizeof(SlotCtl));
        std::memset(B.counters, 0, kCntCount * sizeof(unsigned long long));
        CK(cudaEventCreate(&B.k0));
        CK(cudaEventCreate(&B.k1));
        CK(cudaEventCreateWithFlags(&B.done, cudaEventDisableTiming));
    }
    e->slot_req.assign(R, 0);
    EngineDev &d = e->dev;
    d.slots = e->d_slots;
    d.ctl = e->d_ctl;
    d.caps = e->d_caps;
    d.act_list = e->d_act;
    d.preempt = e->d_preempt;
    d.vacate = e->d_vacate;
    d.strict = e->d_vacate + kNumKinds;
    d.claim_warps = e->d_vacate + kNumKinds + 1;
    d.chunk_now = e->d_vacate + kNumKinds + 2;
    d.act_count = e->d_act_count;
    d.warp_kind = e->d_warp_kind;
    d.warp_cursor = e->d_warp_cursor;
    d.counters = e->d_counters;
    d.chunk_blocks = e->chunk_blocks;
    d.max_requests = R;
    d.n_lanes = e->lanes;
    CK(cudaStreamSynchronize(e->stream));
    if (cfg.use_graph)
        for (IterIO &B : e->iters) {
            fpt_status st = capture_graph(e, B);
            if (st != FPT_OK) return st;
        }
    if (cfg.service_thread) e->service = std::thread(service_loop, e);
    return FPT_OK;
}

Request *find(fpt_engine *e, uint64_t id) {
    auto it = e->reqs.find(id);
    if (it == e->reqs.end() || it->second->released) return nullptr;
    return it->second.get();
}

}  // namespace

extern "C" fpt_status fpt_create(const fpt_engine_config *config, fpt_engine **out) {
    if (!out) return fail(nullptr, FPT_EINVAL, "out is NULL");
    *out = nullptr;
    auto *e = new (std::nothrow) fpt_engine();
    if (!e) return fail(nullptr, FPT_ENOMEM, "host allocation failed");
    const fpt_status st = create_impl(config, e);
    if (st != FPT_OK) {
        set_error(e->error);
        destroy_all(e);
        delete e;
        return st;
    }
    *out = e;
    return FPT_OK;
}

// Validate and queue a request; `payload` (checkpoint bytes) is attached before it becomes
// visible to the admission path.
static fpt_status submit_impl(fpt_engine *e, const fpt_params *params, uint64_t n_traj,
                              uint64_t seed, uint64_t *req_id, std::vector<uint8_t> *payload) {
    if (!e || !params || !req_id) return fail(e, FPT_EINVAL, "NULL argument");
    auto R = std::make_unique<Request>();
    std::string err;
    if (!decode(params, &R->dec, &err)) return fail(e, FPT_EINVAL, err);
    if (params->precision != FPT_FP32)
        return fail(e, FPT_EINVAL, "the engine integrates FP32; use fpt_plain_launch for FP64");
    if (n_traj < 1 || n_traj > (1ull << 40)) return fail(e, FPT_EINVAL, "n_traj must be in [1, 2^40]");
    R->params = *params;
    R->n_traj = n_traj;
    R->seed = seed;
    R->stop_block = params->stop_block ? params->stop_block : 4096;
    const uint64_t nb = (n_traj + R->stop_block - 1) / R->stop_block;
    if (nb > 0xFFFFFFFFull) return fail(e, FPT_EINVAL, "too many id blocks");
    R->n_idblocks = static_cast<uint32_t>(nb);
    if (request_bytes(*params, n_traj, R->stop_block, e->lanes) > e->budget)
        return fail(e, FPT_ENOMEM, "request larger than the engine's memory budget");
    if (payload) R->restore.swap(*payload);
    R->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(e->mu);
        if (e->broken) return fail(e, FPT_ECUDA, "engine is in an error state: " + e->error);
        if (e->pending.size() >= (1u << 20)) return fail(e, FPT_EFULL, "submission queue full");
        R->id = e->next_id++;
        *req_id = R->id;
        e->pending.push_back(R->id);
        e->reqs[R->id] = std::move(R);
    }
    e->cv_work.notify_all();
    return FPT_OK;
}

extern "C" fpt_status fpt_submit(fpt_engine *e, const fpt_params *params, uint64_t n_traj,
                                 uint64_t seed, uint64_t *req_id) {
    return submit_impl(e, params, n_traj, seed, req_id, nullptr);
}

extern "C" fpt_status fpt_step(fpt_engine *e, int n_iterations) {
    if (!e) return fail(e, FPT_EINVAL, "NULL engine");
    if (e->cfg.service_thread) return fail(e, FPT_EBUSY, "a service thread drives this engine");
    std::lock_guard<std::mutex> dk(e->drive_mu);
    CK(cudaSetDevice(e->device));
    for (int i = 0; i < n_iterations; ++i) {
        const fpt_status st = iteration(e);
        if (st != FPT_OK) return st;
    }
    return drain(e);
}

extern "C" fpt_status fpt_poll(fpt_engine *e, uint64_t req_id, fpt_result *out) {
    if (!e || !out) return fail(e, FPT_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(e->mu);
    Request *R = find(e, req_id);
    if (!R) return fail(e, FPT_ENOTFOUND, "unknown request id");
    if (R->phase == kFinished) {
        *out = R->result;
        return FPT_OK;
    }
    std::memset(out, 0, sizeof(*out));
    out->state = FPT_PENDING;
    if (R->slot >= 0 && fresh(e, *R)) {
        const SlotCtl &C = e->h_ctl[R->slot];
        out->n_used = C.n_done;
        out->n_escaped = C.n_esc;
        out->n_censored = C.n_done - C.n_esc;
    }
    out->latency_s = std::chrono::duration<double>(Clock::now() - R->t_submit).count();
    if (e->broken) return fail(e, FPT_ECUDA, "engine is in an error state: " + e->error);
    return FPT_PENDING;
}

extern "C" fpt_status fpt_wait(fpt_engine *e, uint64_t req_id, double timeout_s, fpt_result *out) {
    if (!e || !out) return fail(e, FPT_EINVAL, "NULL argument");
    const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                             std::chrono::duration<double>(timeout_s));
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(e->mu);
            Request *R = find(e, req_id);
            if (!R) return fail(e, FPT_ENOTFOUND, "unknown request id");
            if (R->phase == kFinished) {
                *out = R->result;
                return FPT_OK;
            }
            if (e->broken) return fail(e, FPT_ECUDA, "engine is in an error state: " + e->error);
            if (Clock::now() >= deadline) return fail(e, FPT_ETIMEDOUT, "timed out");
            if (e->cfg.service_thread) {
                e->cv_done.wait_until(lk, deadline);
                continue;
            }
        }
        std::lock_guard<std::mutex> dk(e->drive_mu);
        cudaSetDevice(e->device);
        const fpt_status st = iteration(e);
        if (st != FPT_OK) return st;
    }
}

extern "C" fpt_status fpt_histogram(fpt_engine *e, uint64_t req_id, uint64_t *counts, int nbins,
                                    uint64_t *under, uint64_t *over) {
    if (!e || !counts) return fail(e, FPT_EINVAL, "NULL argument");
    unsigned prefix;
    unsigned *hist;
    {
        std::lock_guard<std::mutex> lk(e->mu);
        Request *R = find(e, req_id);
        if (!R) return fail(e, FPT_ENOTFOUND, "unknown request id");
        if (R->phase != kFinished) return fail(e, FPT_PENDING, "request not finished");
        if (nbins != R->params.hist_bins) return fail(e, FPT_EINVAL, "nbins != params.hist_bins");
        // rows of the result: the id blocks of the prefix, or every row without a stop rule
        prefix = R->params.stop_rse > 0.0 ? R->prefix
                                          : static_cast<unsigned>(hist_rows(R->params, R->n_traj, R->stop_block));
        hist = R->hist;
        if (under) *under = R->sums.under;
        if (over) *over = R->sums.over;
    }
    std::vector<unsigned> rows(static_cast<size_t>(prefix) * nbins);
    CK(cudaSetDevice(e->device));
    if (!rows.empty()) {
        CK(cudaMemcpyAsync(rows.data(), hist, rows.size() * 4, cudaMemcpyDeviceToHost, e->io));
        CK(cudaStreamSynchronize(e->io));
    }
    std::fill(counts, counts + nbins, 0ull);
    for (unsigned p = 0; p < prefix; ++p)
        for (int b = 0; b < nbins; ++b) counts[b] += rows[static_cast<size_t>(p) * nbins + b];
    return FPT_OK;
}

extern "C" fpt_status fpt_request_sums(fpt_engine *e, uint64_t req_id, fpt_sums *out) {
    if (!e || !out) return fail(e, FPT_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(e->mu);
    Request *R = find(e, req_id);
    if (!R) return fail(e, FPT_ENOTFOUND, "unknown request id");
    if (R->phase != kFinished) return fail(e, FPT_PENDING, "request not finished");
    *out = R->sums;
    return FPT_OK;
}

static fpt_status per_traj_impl(fpt_engine *e, uint64_t req_id, int64_t *steps, double *xs,
                                uint64_t n) {
    long long *src;
    Decoded d;
    {
        std::lock_guard<std::mutex> lk(e->mu);
        Request *R = find(e, req_id);
        if (!R) return fail(e, FPT_ENOTFOUND, "unknown request id");
        if (R->phase != kFinished) return fail(e, FPT_PENDING, "request not finished");
        if (!R->per_traj) return fail(e, FPT_EINVAL, "request was submitted without keep_per_traj");
        if (n > R->n_traj) return fail(e, FPT_EINVAL, "n exceeds n_traj");
        src = R->per_traj;
        d = R->dec;
    }
    std::vector<int64_t> tmp;
    int64_t *dst = steps;
    if (!dst) {
        tmp.resize(n);
        dst = tmp.data();
    }
    CK(cudaSetDevice(e->device));
    if (n) {
        CK(cudaMemcpyAsync(dst, src, n * 8, cudaMemcpyDeviceToHost, e->io));
        CK(cudaStreamSynchronize(e->io));
    }
    if (xs)
        for (uint64_t i = 0; i < n; ++i)
            xs[i] = dst[i] < 0 ? (d.output == FPT_OUT_TIME ? -1.0 : NAN)
                               : observable(d, static_cast<uint64_t>(dst[i]));
    return FPT_OK;
}

extern "C" fpt_status fpt_per_traj(fpt_engine *e, uint64_t req_id, double *out, uint64_t n) {
    if (!e || (!out && n)) return fail(e, FPT_EINVAL, "NULL argument");
    return per_traj_impl(e, req_id, nullptr, out, n);
}

extern "C" fpt_status fpt_per_traj_steps(fpt_engine *e, uint64_t req_id, int64_t *out, uint64_t n) {
    if (!e || (!out && n)) return fail(e, FPT_EINVAL, "NULL argument");
    return per_traj_impl(e, req_id, out, nullptr, n);
}

// Bytes of a checkpoint of R: header, control block, accumulators, histogram rows,
// per-trajectory steps (if kept) and at most the ring's capacity of suspended trajectories.
static size_t ckpt_bound(const Request &R, unsigned lanes) {
    size_t b = sizeof(CkptHeader) + sizeof(SlotCtl) + R.n_idblocks * sizeof(IdBlockAcc) +
               hist_rows(R.params, R.n_traj, R.stop_block) * R.params.hist_bins * 4 +
               static_cast<size_t>(park_capacity(R.n_traj, lanes)) * sizeof(ParkEntry);
    if (R.params.keep_per_traj) b += R.n_traj * 8;
    return b;
}

extern "C" fpt_status fpt_checkpoint(fpt_engine *e, uint64_t req_id, void *buf, size_t *size) {
    if (!e || !size) return fail(e, FPT_EINVAL, "NULL argument");
    {
        std::lock_guard<std::mutex> lk(e->mu);
        Request *R = find(e, req_id);
        if (!R) return fail(e, FPT_ENOTFOUND, "unknown request id");
        if (R->phase == kFinished || R->phase == kCancelled)
            return fail(e, FPT_EINVAL, "request already finished or cancelled");
        const size_t bound = ckpt_bound(*R, e->lanes);
        if (!buf) {
            *size = bound;
            return FPT_OK;
        }
        if (*size < bound) return fail(e, FPT_EINVAL, "checkpoint buffer too small");
        R->suspending = true;
    }
    e->cv_work.notify_all();
    // wait until the request's lanes have suspended (drive the engine without a service thread)
    for (int it = 0; it < 1000; ++it) {
        {
            std::unique_lock<std::mutex> lk(e->mu);
            Request *R = find(e, req_id);
            if (!R) return fail(e, FPT_ENOTFOUND, "request vanished");
            if (R->quiesced || R->phase == kPending || R->phase == kFinished) break;
            if (e->broken) return fail(e, FPT_ECUDA, "engine is in an error state: " + e->error);
            if (e->cfg.service_thread) {
                e->cv_done.wait_for(lk, std::chrono::milliseconds(100));
                continue;
            }
        }
        std::lock_guard<std::mutex> dk(e->drive_mu);
        cudaSetDevice(e->device);
        const fpt_status st = iteration(e);
        if (st != FPT_OK) return st;
    }
    std::lock_guard<std::mutex> dk(e->drive_mu);   // no launch may run while we read
    CK(cudaSetDevice(e->device));
    {
        const fpt_status ds = drain(e);
        if (ds != FPT_OK) return ds;
    }
    std::lock_guard<std::mutex> lk(e->mu);
    Request *R = find(e, req_id);
    if (!R) return fail(e, FPT_ENOTFOUND, "request vanished");
    uint8_t *q = static_cast<uint8_t *>(buf);
    CkptHeader H{};
    H.magic = kCkptMagic;
    H.version = kCkptVersion;
    H.params = R->params;
    H.n_traj = R->n_traj;
    H.seed = R->seed;
    H.stop_block = R->stop_block;
    H.n_idblocks = R->n_idblocks;
    H.has_per_traj = R->params.keep_per_traj ? 1 : 0;
    SlotCtl C{};
    if (R->phase == kPending) {
        H.n_park = 0;
    } else if (!R->quiesced) {
        return fail(e, FPT_ETIMEDOUT, "request did not quiesce");
    } else {
        CK(cudaMemcpy(&C, e->d_ctl + R->slot, sizeof(SlotCtl), cudaMemcpyDeviceToHost));
        H.n_park = C.park_tail - C.park_head;
    }
    const size_t nb = R->n_idblocks,
                 hist_b = hist_rows(R->params, R->n_traj, R->stop_block) * static_cast<size_t>(R->params.hist_bins) * 4;
    std::memcpy(q, &H, sizeof(H));
    q += sizeof(H);
    std::memcpy(q, &C, sizeof(C));
    q += sizeof(C);
    if (R->phase == kPending) {
        std::memset(q, 0, nb * sizeof(IdBlockAcc) + hist_b + (H.has_per_traj ? R->n_traj * 8 : 0));
        q += nb * sizeof(IdBlockAcc) + hist_b;
        if (H.has_per_traj) {
            std::memset(q, 0xFF, R->n_traj * 8);
            q += R->n_traj * 8;
        }
    } else {
        CK(cudaMemcpy(q, R->acc, nb * sizeof(IdBlockAcc), cudaMemcpyDeviceToHost));
        q += nb * sizeof(IdBlockAcc);
        CK(cudaMemcpy(q, R->hist, hist_b, cudaMemcpyDeviceToHost));
        q += hist_b;
        if (H.has_per_traj) {
            CK(cudaMemcpy(q, R->per_traj, R->n_traj * 8, cudaMemcpyDeviceToHost));
            q += R->n_traj * 8;
        }
        for (unsigned i = 0; i < H.n_park; ++i) {
            const unsigned idx = (C.park_head + i) % R->park_cap;
            CK(cudaMemcpy(q, R->park + idx, sizeof(ParkEntry), cudaMemcpyDeviceToHost));
            q += sizeof(ParkEntry);
        }
    }
    *size = static_cast<size_t>(q - static_cast<uint8_t *>(buf));
    // release: the slot is freed after the device state says no lane holds it
    R->released = true;
    if (R->phase == kPending) {
        e->pending.erase(std::find(e->pending.begin(), e->pending.end(), req_id));
        e->reqs.erase(req_id);
    } else {
        R->phase = kCancelled;
        static const int cancelled = kSlotCancelled;
        CK(cudaMemcpy(&e->d_ctl[R->slot].state, &cancelled, sizeof(int), cudaMemcpyHostToDevice));
    }
    return FPT_OK;
}

extern "C" fpt_status fpt_restore(fpt_engine *e, const void *buf, size_t size, uint64_t *req_id) {
    if (!e || !buf || !req_id) return fail(e, FPT_EINVAL, "NULL argument");
    if (size < sizeof(CkptHeader) + sizeof(SlotCtl)) return fail(e, FPT_EINVAL, "checkpoint too short");
    CkptHeader H;
    std::memcpy(&H, buf, sizeof(H));
    if (H.magic != kCkptMagic || H.version != kCkptVersion) return fail(e, FPT_EINVAL, "not a checkpoint");
    // the header's sizes must be those a request of these parameters has, before any of them
    // is used to size a copy
    {
        Decoded d;
        std::string err;
        if (!decode(&H.params, &d, &err)) return fail(e, FPT_EINVAL, "checkpoint parameters: " + err);
    }
    const uint32_t B = H.params.stop_block ? H.params.stop_block : 4096;
    if (H.n_traj < 1 || H.n_traj > (1ull << 40) || H.stop_block != B ||
        H.n_idblocks != (H.n_traj + B - 1) / B || H.n_park > H.n_traj || H.has_per_traj > 1 ||
        H.has_per_traj != static_cast<uint64_t>(H.params.keep_per_traj != 0))
        return fail(e, FPT_EINVAL, "checkpoint header is inconsistent");
    const size_t nb = H.n_idblocks;
    const size_t want = sizeof(CkptHeader) + sizeof(SlotCtl) + nb * sizeof(IdBlockAcc) +
                        hist_rows(H.params, H.n_traj, B) * static_cast<size_t>(H.params.hist_bins) * 4 +
                        (H.has_per_traj ? H.n_traj * 8 : 0) + H.n_park * sizeof(ParkEntry);
    if (size != want) return fail(e, FPT_EINVAL, "checkpoint size does not match its header");
    if (H.n_park > park_capacity(H.n_traj, e->lanes))
        return fail(e, FPT_EINVAL, "checkpoint holds more suspended trajectories than this engine's ring");
    std::vector<uint8_t> payload(static_cast<const uint8_t *>(buf), static_cast<const uint8_t *>(buf) + size);
    return submit_impl(e, &H.params, H.n_traj, H.seed, req_id, &payload);
}

extern "C" fpt_status fpt_release(fpt_engine *e, uint64_t req_id) {
    if (!e) return fail(e, FPT_EINVAL, "NULL engine");
    std::lock_guard<std::mutex> lk(e->mu);
    Request *R = find(e, req_id);
    if (!R) return fail(e, FPT_ENOTFOUND, "unknown request id");
    R->released = true;
    if (R->phase == kPending) {
        e->pending.erase(std::find(e->pending.begin(), e->pending.end(), req_id));
        e->reqs.erase(req_id);
        return FPT_OK;
    }
    if (R->phase == kRunning) {
        // lanes drop the request at the start of the next launch
        R->phase = kCancelled;
        static const int cancelled = kSlotCancelled;
        cudaSetDevice(e->device);
        const cudaError_t ce = cudaMemcpy(&e->d_ctl[R->slot].state, &cancelled, sizeof(int),
                                          cudaMemcpyHostToDevice);
        if (ce != cudaSuccess) {
            e->broken = true;
            return fail(e, FPT_ECUDA, std::string("cancel: ") + cudaGetErrorString(ce));
        }
        return FPT_OK;
    }
    if (R->slot < 0) {   // finished and its slot already recycled
        free_request_buffers(*R, e);
        e->reqs.erase(req_id);
    }
    return FPT_OK;
}

extern "C" fpt_status fpt_get_counters(fpt_engine *e, fpt_engine_counters *out) {
    if (!e || !out) return fail(e, FPT_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(e->mu);
    std::memset(out, 0, sizeof(*out));
    out->iterations = e->iterations;
    out->useful_steps = e->h_counters[kCntUseful];
    out->escapes = e->h_counters[kCntEscapes];
    out->censored = e->h_counters[kCntCensored];
    out->check_flags = e->h_counters[kCntCheck];
    out->lane_step_slots = e->lane_slots;
    out->lanes = e->lanes;
    out->grid = e->grid;
    out->block = e->block;
    out->traj_per_thread = e->T;
    out->chunk_steps = e->chunk_blocks * kBlockSteps;
    out->kernel_ms = e->kernel_ms;
    out->preempted = e->preempted;
    for (int s = 0; s < e->maxr; ++s)
        if (e->slot_req[s]) ++out->resident_requests;
    out->pending_requests = static_cast<uint32_t>(e->pending.size());
    return FPT_OK;
}

extern "C" fpt_status fpt_engine_occupancy(int32_t traj_per_thread, int32_t threads_per_block,
                                           int32_t *blocks_per_sm) {
    if (!blocks_per_sm) return fail(nullptr, FPT_EINVAL, "blocks_per_sm is NULL");
    *blocks_per_sm = 0;
    if (traj_per_thread != 1 && traj_per_thread != 2)
        return fail(nullptr, FPT_EINVAL, "traj_per_thread must be 1 or 2");
    const int max_block = traj_per_thread == 1 ? 640 : 256;
    if (threads_per_block < 32 || threads_per_block % 32 || threads_per_block > max_block)
        return FPT_OK;   // the kernel cannot launch with this shape: 0 CTAs per SM
    int bps = 0;
    const cudaError_t ce = engine_chunk_occupancy(traj_per_thread, threads_per_block, &bps);
    if (ce != cudaSuccess) return fail(nullptr, FPT_ECUDA, std::string("occupancy: ") + cudaGetErrorString(ce));
    *blocks_per_sm = bps;
    return FPT_OK;
}

extern "C" void *fpt_engine_stream(fpt_engine *e) { return e ? static_cast<void *>(e->stream) : nullptr; }

extern "C" fpt_status fpt_destroy(fpt_engine *e) {
    if (!e) return fail(e, FPT_EINVAL, "NULL engine");
    destroy_all(e);
    delete e;
    return FPT_OK;
}

extern "C" const char *fpt_last_error(fpt_engine *e) {
    if (e) return t_engine_error.empty() ? e->error.c_str() : t_engine_error.c_str();
    return get_error().c_str();
}
