// engine_kernels.cu -- the persistent batched FPT kernel and the completion scan.
//
// One launch ("chunk") advances the resident lanes by the launch's blocks of kBlockSteps steps
// per warp on average (chunk_blocks, or fewer while a small request is new; Euler-Maruyama or
// stochastic Heun; the last quarter of the blocks is a per-CTA pool, so the warps of an SM
// finish together).  A lane integrates one trajectory:
// Philox4x32-10 -> Box-Muller -> step (Alg. 1 / 3) on a phase wrapped to [-pi, pi) with an
// integer winding count.  Escape and upper-wrap events are caught by one running maximum per
// block (exact replay of the rare block that reached a bound); the lower wrap (r < -pi) is
// applied at the end of each block.  At the block end the warp votes, finished lanes publish
// their exact result (grouped in the warp, additions nobody waits for) and the warp refills them
// -- with suspended trajectories, then ids of its reservoir, then new ids from the requests'
// work queues (one atomic per claim) -- so lanes never wait for the slowest trajectory of a
// batch (the dynamic job assignment of Sec. III.B, Fig. 6).
//
// Preemption: at the end of a launch, lanes of requests above their fair share may suspend
// their trajectory into the request's ring (state r, v, w, step count, id); a later refill
// resumes it exactly.  The ramped bias is formed from the trajectory's own step count, so a
// trajectory's arithmetic never depends on which lane, launch or schedule ran it.
//
// A warp integrates one kind at a time (model x integrator x constant or ramped bias: eight
// code paths); the request of each lane is free, so requests of the same kind share warps.
// Refill is round-robin over the claimable requests; while some request is starved, each is
// kept within a fair-share cap on the lanes it holds, otherwise no lane idles while any request
// has work.
#include <cstdint>

#include "engine_dev.h"
#include "fpt_device.cuh"
#include "internal.h"

namespace fpt {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

struct Lane {
    float r, v, hb;
    int w, slot, esc;
    unsigned c_lo, c_hi, gid_lo, gid_hi;
    unsigned budget;      // blocks to the next event: step budget end, bias re-base, carry
    float gb, Jf;         // bias base and 4 x blocks since the base (exact)
    float dt, A, amp, bmc, nudt;
    PhiloxLane P;         // the trajectory's Philox stream (round keys, fixed words of rounds 0-2)
};

__device__ __forceinline__ float qnan_f() { return __int_as_float(0x7FFFFFFF); }

// Bounds checks of the FPT_CHECK build: a violated one sets its bit in the global check word
// (counters[kCntCheck], read back with the engine counters) and the access is skipped; nothing
// traps.  In the regular build every check is `true`.
enum : unsigned {
    kChkSlot = 0,      // request slot outside [0, max_requests)
    kChkLane = 1,      // lane-state index outside [0, n_lanes)
    kChkIdBlock = 2,   // id block outside [0, n_idblocks)
    kChkHistRow = 3,   // histogram row outside [0, hist_rows)
    kChkBin = 4,       // histogram bin outside [0, hist_bins)
    kChkTraj = 5,      // trajectory index outside [0, n_traj)
    kChkPark = 6,      // suspended-trajectory ring index outside [0, park_cap)
    kChkKind = 7,      // kind outside [0, kNumKinds)
};
#ifdef FPT_CHECK
__device__ __forceinline__ bool checked(const EngineDev &E, bool ok, unsigned bit) {
    if (!ok) atomicOr(&E.counters[kCntCheck], 1ull << bit);
    return ok;
}
#else
__device__ __forceinline__ constexpr bool checked(const EngineDev &, bool, unsigned) { return true; }
#endif

template <typename V>
__device__ __forceinline__ V vload(const V &x) {
    return *const_cast<const volatile V *>(&x);
}

__device__ __forceinline__ void set_idle(Lane &L) {
    L.slot = -1;
    L.r = qnan_f();
    L.v = 0.0f;
    L.hb = 0.0f;
    L.esc = -1;
    L.budget = 0xFFFFFFFFu;
    L.dt = L.A = L.amp = L.bmc = L.nudt = L.gb = L.Jf = 0.0f;
}

__device__ __forceinline__ unsigned clamp_u32(unsigned long long x) {
    return x > 0xFFFFFFFFull ? 0xFFFFFFFFu : static_cast<unsigned>(x);
}

// Request constants and the trajectory's Philox stream; gid and the block count c are set.
__device__ __forceinline__ void load_consts(Lane &L, const SlotDev *S) {
    L.dt = S->dt;
    L.A = S->A;
    L.amp = S->amp;
    L.bmc = S->bmc;
    L.nudt = S->nudt;
    philox_lane_init(L.P, S->key0, S->key1, L.c_hi, L.gid_lo, L.gid_hi);
}

__device__ __forceinline__ unsigned long long lane_c(const Lane &L) {
    return (static_cast<unsigned long long>(L.c_hi) << 32) | L.c_lo;
}

// Bias base and event countdown from the trajectory's Philox block count c (4 steps each; c is
// a multiple of kBlockPhilox at block boundaries):
// gb = gamma0 + nu dt 4 c_base (FP64, rounded once), Jf = 4 (c - c_base),
// budget = kernel blocks until the step budget ends, the next re-base or the next carry of the
// low 32-bit word of c, whichever is first (the high word is only updated at that event).
__device__ __forceinline__ void set_progress(Lane &L, const SlotDev *S) {
    const unsigned long long c = lane_c(L);
    const unsigned long long cb = c - (c % kRebaseBlocks);
    L.gb = static_cast<float>(S->gamma0 + S->nudt_d * static_cast<double>(4ull * cb));
    L.Jf = static_cast<float>(4ull * (c - cb));
    const unsigned long long to_end = S->nblocks > c ? S->nblocks - c : 0ull;
    const unsigned long long to_base = kRebaseBlocks - (c - cb);
    const unsigned long long to_carry = 0x100000000ull - (c & 0xFFFFFFFFull);
    unsigned long long m = to_end < to_base ? to_end : to_base;
    m = m < to_carry ? m : to_carry;
    L.budget = static_cast<unsigned>((m + kBlockPhilox - 1) / kBlockPhilox);
}

// Start trajectory `idx` of request slot s.
__device__ __forceinline__ void init_lane(Lane &L, const EngineDev &E, int s, unsigned long long idx) {
    const SlotDev *S = E.slots + s;
    const unsigned long long gid = S->traj_offset + idx;
    L.slot = s;
    L.gid_lo = static_cast<unsigned>(gid);
    L.gid_hi = static_cast<unsigned>(gid >> 32);
    L.c_lo = L.c_hi = 0;
    L.r = S->r0;
    L.v = S->v0;
    L.w = S->w0;
    L.hb = fminf(S->eb0, kPiF);
    L.esc = -1;
    load_consts(L, S);
    L.gb = S->gb0;       // set_progress at c = 0, formed on the host
    L.Jf = 0.0f;
    L.budget = S->budget0;
}

// Continue a suspended trajectory exactly where it stopped.
__device__ __forceinline__ void resume_lane(Lane &L, const EngineDev &E, int s, const ParkEntry &P) {
    const SlotDev *S = E.slots + s;
    L.slot = s;
    L.r = P.r;
    L.v = P.v;
    L.w = P.w;
    L.c_lo = P.c_lo;
    L.c_hi = P.c_hi;
    L.gid_lo = P.gid_lo;
    L.gid_hi = P.gid_hi;
    L.hb = fminf(fmaf(-kTwoPiF, static_cast<float>(P.w - S->w0), S->eb0), kPiF);
    L.esc = -1;
    load_consts(L, S);
    set_progress(L, S);
}

// Histogram bin of x = out_a + out_b k (IEEE double, separately rounded): -1 below the range,
// hist_bins above it.
__device__ __forceinline__ int hist_bin(const SlotDev *S, unsigned long long k) {
    const double kd = static_cast<double>(k);
    const double x = S->output == FPT_OUT_TIME ? __dmul_rn(S->out_b, kd)
                                               : __dadd_rn(S->out_a, __dmul_rn(S->out_b, kd));
    if (x < S->hist_lo) return -1;
    if (x >= S->hist_hi) return S->hist_bins;
    const int bin = static_cast<int>(floor(__dmul_rn(__dsub_rn(x, S->hist_lo), S->hist_inv_w)));
    return bin < S->hist_bins ? bin : S->hist_bins - 1;
}

// Per-CTA view of the requests during one launch (shared memory), set up at kernel start:
//   ok[s]   bit 0: request s has ids left to claim, bit 1: it has suspended trajectories to
//           resume (both as of the launch start; cleared when a warp finds them exhausted),
//   held[s] lanes of this CTA that hold a trajectory of s (the CTA's share of the fair-share
//           cap is checked against it, so claims need no global read),
//   budget[s] reservoir ids this CTA may hold for s: its share of the room the request's ring
//           had at launch start beyond one slot per lane (kept for suspensions), so that the
//           reservoirs returned to the ring at the end of the launch always fit.
struct CtaView {
    unsigned *ok;
    int *held;
    int *budget;                 // ids this CTA's warps may still hold in reservoirs, per request
    int *res_slot, *res_cnt;     // per warp of the CTA: reservoir request and count ...
    unsigned long long *res_base;   // ... and first id (ids res_base .. res_base + res_cnt - 1)
    int *started;                // per warp: trajectories it started in this launch
    int *pool;                   // blocks of this launch not yet taken by a warp of the CTA
};

// Publish the trajectories finishing in this warp at this block end (warp-collective: every lane
// calls it, `fin` says whether its trajectory finished).  Lanes are grouped by (request slot, id
// block) with a match; each group's counts and the 32-bit limbs of k and k^2 are gathered by
// shuffles, and its first lane adds them into the id block with atomic additions whose result
// it does not wait for, and gives back the group's in-flight places.  Histogram counts are
// grouped by (slot, id block, bin) the same way.  The scan kernel reads the id blocks only
// after the launch, so the order of the additions is free.
__device__ __forceinline__ void emit_warp(const EngineDev &E, const CtaView &V, bool fin, int slot,
                                          unsigned long long gid, bool escaped, unsigned long long k) {
    const int lane = threadIdx.x & 31;
    // an index out of range (checked build only) drops the trajectory's result
    if (fin) fin = checked(E, slot >= 0 && slot < E.max_requests, kChkSlot);
    if (!__any_sync(kFull, fin)) return;   // an event block without a finished trajectory
    const SlotDev *S = E.slots + (fin ? slot : 0);
    unsigned long long idx = 0;
    unsigned ib = 0, row = 0;
    int bin = -2;
    if (fin) {
        idx = gid - S->traj_offset;
        ib = static_cast<unsigned>(id_block_quot(idx, S->ib_magic, S->ib_shift));
        row = S->hist_per_block ? ib : static_cast<unsigned>(idx / kHistRowIds);
        if (escaped) bin = hist_bin(S, k);
        fin = checked(E, idx < S->n_traj, kChkTraj) && checked(E, ib < S->n_idblocks, kChkIdBlock) &&
              checked(E, row < S->hist_rows, kChkHistRow) &&
              checked(E, bin == -2 || (bin >= -1 && bin <= S->hist_bins), kChkBin);
        if (fin && S->per_traj) S->per_traj[idx] = escaped ? static_cast<long long>(k) : -1ll;
    }
    // slot < 2^10, id block and row < 2^32, bin < 2^21: distinct keys for distinct groups
    const unsigned long long gkey = fin ? (static_cast<unsigned long long>(slot) << 32) | ib : ~0ull;
    const unsigned grp = __match_any_sync(kFull, gkey);
    const unsigned long long bkey =
        fin && bin >= 0 && bin < S->hist_bins
            ? (static_cast<unsigned long long>(slot) << 53) | (static_cast<unsigned long long>(row) << 21) |
                  static_cast<unsigned long long>(bin)
            : ~0ull;
    const unsigned bgrp = __match_any_sync(kFull, bkey);
    if (!fin) return;
    IdBlockAcc *A = S->acc + ib;
    if (bkey != ~0ull && lane == __ffs(bgrp) - 1)
        atomicAdd(S->hist + static_cast<size_t>(row) * S->hist_bins + bin, static_cast<unsigned>(__popc(bgrp)));
    // limbs: k = k0 + 2^32 k1, k^2 = q0 + 2^32 q1 + 2^64 q2 (each < 2^32)
    const unsigned long long kk_lo = escaped ? k * k : 0ull, kk_hi = escaped ? __umul64hi(k, k) : 0ull;
    const unsigned long long ke = escaped ? k : 0ull;
    unsigned long long l[5] = {ke & 0xFFFFFFFFull, ke >> 32, kk_lo & 0xFFFFFFFFull, kk_lo >> 32, kk_hi};
    unsigned cnt = (escaped ? 1u : 0u) | (bin == -1 ? 2u : 0u) | (escaped && bin == S->hist_bins ? 4u : 0u);
    unsigned n_e = cnt & 1u, n_u = (cnt >> 1) & 1u, n_o = cnt >> 2;
    const int leader = __ffs(grp) - 1;
    unsigned rest = grp & ~(1u << leader);
    while (rest) {   // every lane of the group runs the same sequence of shuffles
        const int src = __ffs(rest) - 1;
        rest &= rest - 1u;
        const unsigned c = __shfl_sync(grp, cnt, src);
        unsigned long long m[5];
#pragma unroll
        for (int j = 0; j < 5; ++j) m[j] = __shfl_sync(grp, l[j], src);   // src's l is unchanged
        if (lane == leader) {
            n_e += c & 1u;
            n_u += (c >> 1) & 1u;
            n_o += c >> 2;
#pragma unroll
            for (int j = 0; j < 5; ++j) l[j] += m[j];
        }
    }
    if (lane != leader) return;
    if (n_e) {
        atomicAdd(&A->escaped, n_e);
        atomicAdd(&A->s1[0], l[0]);
        if (l[1]) atomicAdd(&A->s1[1], l[1]);
        atomicAdd(&A->s2[0], l[2]);
        if (l[3]) atomicAdd(&A->s2[1], l[3]);
        if (l[4]) atomicAdd(&A->s2[2], l[4]);
    }
    if (n_u) atomicAdd(&A->under, n_u);
    if (n_o) atomicAdd(&A->over, n_o);
    const int n = __popc(grp);
    atomicAdd(&A->done, static_cast<unsigned>(n));
    atomicSub(&E.ctl[slot].inflight, n);
    atomicSub(&V.held[slot], n);
}

// Rare per-lane path: the phase reached hb = min(eb, pi), where eb = phi* - 2 pi w is the
// threshold in the current cell's coordinates.  Escape freezes the lane (NaN phase: no further
// events) and records the step within the block; otherwise wrap upwards and count a winding.
__device__ __forceinline__ void phase_event(Lane &L, const EngineDev &E, int s) {
    const SlotDev *S = E.slots + L.slot;
    const float eb0 = S->eb0;
    const int w0 = S->w0;
    const float eb = fmaf(-kTwoPiF, static_cast<float>(L.w - w0), eb0);
    if (L.r >= eb) {
        L.esc = s;
        L.r = qnan_f();
        return;
    }
    L.r -= kTwoPiF;
    L.w += 1;
    L.hb = fminf(fmaf(-kTwoPiF, static_cast<float>(L.w - w0), eb0), kPiF);
}

// Lower wrap, applied at block ends (sin is accurate a little below -pi in between).
__device__ __forceinline__ void wrap_down(Lane &L, const EngineDev &E) {
    const SlotDev *S = E.slots + L.slot;
    L.r += kTwoPiF;
    L.w -= 1;
    L.hb = fminf(fmaf(-kTwoPiF, static_cast<float>(L.w - S->w0), S->eb0), kPiF);
}

// Finish lanes that escaped in the last block or reached the step budget (warp-collective).
template <int T>
__device__ __forceinline__ void finish_lanes(Lane (&L)[T], const EngineDev &E, const CtaView &V,
                                             unsigned long long &useful, int &n_active, unsigned &n_esc,
                                             unsigned &n_cens) {
#pragma unroll
    for (int t = 0; t < T; ++t) {
        bool fin = false, escaped = false;
        unsigned long long k = 0;
        if (L[t].slot < 0) {
            L[t].budget = 0xFFFFFFFFu;
        } else if (L[t].esc >= 0 || L[t].budget == 0) {
            const SlotDev *S = E.slots + L[t].slot;
            const unsigned long long c = lane_c(L[t]);
            const unsigned long long max_steps = S->max_steps;
            if (L[t].esc < 0 && c < S->nblocks) {   // re-base of the bias, not the end of the budget
                set_progress(L[t], S);
            } else {
                fin = true;
                if (L[t].esc >= 0) {
                    k = 4ull * (c - kBlockPhilox) + static_cast<unsigned long long>(L[t].esc) + 1ull;
                    escaped = k <= max_steps;
                }
                if (escaped) useful -= static_cast<unsigned long long>(kBlockSteps - 1 - L[t].esc);
                else useful -= 4ull * c - max_steps;
            }
        }
        const unsigned long long gid = (static_cast<unsigned long long>(L[t].gid_hi) << 32) | L[t].gid_lo;
        emit_warp(E, V, fin, L[t].slot, gid, escaped, k);
        if (fin) {
            if (escaped) ++n_esc;
            else ++n_cens;
            set_idle(L[t]);
            --n_active;
        }
    }
}

// Warp-collective refill of idle lanes with trajectories of requests of kind `kind`.  Lane 0
// takes, per request in round-robin order, suspended trajectories first, then ids from the
// warp's reservoir, then new ids from the request's queue head: one atomic addition on the head
// per claim, claiming up to kReserveIds more for the reservoir when it is empty and the CTA's
// budget allows, and the in-flight count raised by what was actually started (an addition
// nobody waits for).  While some request is
// starved (strict caps, set by the host with preemption orders) each request is kept within
// this CTA's share of its fair-share cap, counted in shared memory; otherwise lanes take work
// from the first request that has some, so no lane idles while any request has work.
template <int T>
__device__ __forceinline__ void refill(Lane (&L)[T], const EngineDev &E, const CtaView &V, int kind,
                                       int &n_active, unsigned &cursor, unsigned b) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    unsigned idle[T];
    int total = 0;
#pragma unroll
    for (int t = 0; t < T; ++t) {
        idle[t] = __ballot_sync(kFull, L[t].slot < 0);
        total += __popc(idle[t]);
    }
    if (total == 0) return;
    if (static_cast<int>(threadIdx.x >> 5) >= *E.claim_warps) return;   // spread scarce work
    if (!checked(E, kind >= 0 && kind < kNumKinds, kChkKind)) return;
    const int cnt = E.act_count[kind];
    if (cnt <= 0) return;
    const int *list = E.act_list + kind * E.max_requests;
    const bool capped = *E.strict != 0;
    const int wl = static_cast<int>(threadIdx.x >> 5);
    // A warp that holds a reservoir serves its request first, so the reservoir drains.
    __syncwarp();
    const int rs = V.res_slot[wl];
    const bool res_first = V.res_cnt[wl] > 0 && rs >= 0 && rs < E.max_requests && E.slots[rs].kind == kind;
    {
        for (int scanned = res_first ? -1 : 0; scanned < cnt && total > 0; ++scanned) {
            const int s = scanned < 0 ? rs : list[cursor % static_cast<unsigned>(cnt)];
            if (scanned >= 0) ++cursor;
            if (!checked(E, s >= 0 && s < E.max_requests, kChkSlot)) continue;
            unsigned long long base = 0, rb = 0;
            int got = 0, gp = 0, rt = 0;
            unsigned p0 = 0;
            if (lane == 0 && ((V.ok[s] & 3u) || V.res_slot[wl] == s)) {
                SlotCtl *C = E.ctl + s;
                const unsigned long long n_traj = E.slots[s].n_traj;
                int want = total;
                if (capped) {
                    const int cap = (E.caps[s] + static_cast<int>(gridDim.x) - 1) / static_cast<int>(gridDim.x);
                    const int room = cap - V.held[s];
                    want = room < 0 ? 0 : (room < want ? room : want);
                }
                // 1. suspended trajectories
                if (want > 0 && (V.ok[s] & 2u)) {
                    const int pv = atomicSub(&C->park_avail, want);
                    if (pv <= 0) {
                        atomicAdd(&C->park_avail, want);
                        atomicAnd(&V.ok[s], ~2u);
                    } else {
                        gp = pv < want ? pv : want;
                        if (gp < want) atomicAdd(&C->park_avail, want - gp);
                        p0 = atomicAdd(&C->park_head, static_cast<unsigned>(gp));
                        atomicSub(&C->park_used, gp);
                    }
                }
                got = gp;
                // 2. this warp's reservoir of ids claimed earlier
                if (want > got && V.res_slot[wl] == s && V.res_cnt[wl] > 0) {
                    rt = want - got < V.res_cnt[wl] ? want - got : V.res_cnt[wl];
                    rb = V.res_base[wl];
                    V.res_base[wl] += static_cast<unsigned long long>(rt);
                    V.res_cnt[wl] -= rt;
                    atomicAdd(&V.budget[s], rt);
                    got += rt;
                }
                // 3. the queue head, with more for the reservoir when it is free: as many as this
                //    warp is expected to start in the rest of a full launch at its rate so far
                //    (at most kReserveIds, none while caps are enforced), within the CTA's budget;
                //    in a shorter launch the surplus goes back to the ring at its end.
                //    Only warps that start a trajectory at least every 8 blocks keep one: for
                //    long trajectories the ids would mostly return to the ring unused.
                if (want > got && (V.ok[s] & 1u)) {
                    const int wn = want - got;
                    int extra = 0;
                    if (V.res_cnt[wl] == 0 && !capped && b > 0 && 8u * static_cast<unsigned>(V.started[wl]) >= b) {
                        const unsigned long long expect =
                            static_cast<unsigned long long>(V.started[wl]) * (E.chunk_blocks > b ? E.chunk_blocks - b : 0u) / b;
                        const int want_extra = expect < static_cast<unsigned long long>(kReserveIds)
                                                   ? static_cast<int>(expect) : kReserveIds;
                        if (want_extra > 0) {
                            if (atomicSub(&V.budget[s], want_extra) >= want_extra) extra = want_extra;
                            else atomicAdd(&V.budget[s], want_extra);
                        }
                    }
                    const int cl = wn + extra;
                    base = atomicAdd(&C->head, static_cast<unsigned long long>(cl));
                    int keep = 0;
                    if (base < n_traj) {
                        const unsigned long long left = n_traj - base;
                        const int avail = left < static_cast<unsigned long long>(cl) ? static_cast<int>(left) : cl;
                        const int use = avail < wn ? avail : wn;
                        got += use;
                        keep = avail - use;
                        if (keep > 0) {
                            V.res_slot[wl] = s;
                            V.res_base[wl] = base + static_cast<unsigned long long>(use);
                            V.res_cnt[wl] = keep;
                        }
                    }
                    if (extra > keep) atomicAdd(&V.budget[s], extra - keep);
                    if (base + static_cast<unsigned long long>(cl) >= n_traj) atomicAnd(&V.ok[s], ~1u);
                }
                if (got) {
                    atomicAdd(&C->inflight, got);
                    atomicAdd(&V.held[s], got);
                    V.started[wl] += got;
                }
            }
            got = __shfl_sync(kFull, got, 0);
            if (got == 0) continue;
            gp = __shfl_sync(kFull, gp, 0);
            p0 = __shfl_sync(kFull, p0, 0);
            rt = __shfl_sync(kFull, rt, 0);
            rb = __shfl_sync(kFull, rb, 0);
            base = __shfl_sync(kFull, base, 0);
            const SlotDev *S = E.slots + s;
            int before = 0;
#pragma unroll
            for (int t = 0; t < T; ++t) {
                const unsigned m = idle[t];
                const int rank = before + __popc(m & lt);
                if (((m >> lane) & 1u) && rank < got) {
                    if (rank < gp) {
                        const unsigned pi = (p0 + static_cast<unsigned>(rank)) % S->park_cap;
                        if (checked(E, pi < S->park_cap, kChkPark)) resume_lane(L[t], E, s, S->park[pi]);
                    } else if (rank < gp + rt) {
                        init_lane(L[t], E, s, rb + static_cast<unsigned long long>(rank - gp));
                    } else {
                        init_lane(L[t], E, s, base + static_cast<unsigned long long>(rank - gp - rt));
                    }
                    ++n_active;
                }
                before += __popc(m);
                idle[t] = __ballot_sync(kFull, L[t].slot < 0);
            }
            total -= got;
        }
    }
}

// Integrate blocks of kBlockSteps steps with model M, integrator H and bias kind R (constant or
// ramped) until the warp's share of the launch's blocks is done (`limit`, extended from the
// CTA's pool) or the whole warp has run out of work.  Returns the next block index.
// A launch's blocks: each warp first runs (1 - 1/kPoolDiv) of the launch's block count, then
// takes kGrant blocks at a time from its CTA's pool of the rest, so warps whose lanes had more
// events (replays, refills) do fewer blocks and the warps of an SM finish together instead of
// leaving the SM to a few late ones (+3.7 % at 4096-step launches, +0.8 % at 65 536).
constexpr unsigned kPoolDiv = 4;
constexpr int kGrant = 4;

// More blocks for this warp from its CTA's pool (warp-collective); false when the pool is empty.
__device__ __forceinline__ bool grant(const CtaView &V, unsigned &limit) {
    int g = 0;
    if ((threadIdx.x & 31) == 0) {
        const int p = atomicSub(V.pool, kGrant);
        g = p >= kGrant ? kGrant : (p > 0 ? p : 0);
    }
    g = __shfl_sync(kFull, g, 0);
    limit += static_cast<unsigned>(g);
    return g > 0;
}

template <int M, int H, int R, int T>
__device__ __forceinline__ unsigned run_blocks(Lane (&L)[T], const EngineDev &E, const CtaView &V, unsigned b,
                                               int &n_active,
                               unsigned &cursor, unsigned long long &useful, unsigned &n_esc,
                               unsigned &n_cens, unsigned &limit) {
    // Steps are counted when the number of active lanes changes (at events) and at the end:
    // useful += kBlockSteps x active lanes x blocks since the last count.
    unsigned b_count = b;
    // Constant bias (R = 0): the bias line is the same in every block until an event changes the
    // lane (re-base, refill); it is formed here and after each event.
    float gs[T], gsl[T];
#pragma unroll
    for (int t = 0; t < T; ++t)
        if constexpr (!R) bias_line(fmaf(L[t].nudt, L[t].Jf, L[t].gb), L[t].nudt, L[t].dt, gs[t], gsl[t]);
    while (b < limit || grant(V, limit)) {
        // the block's normals: Philox blocks c .. c + kBlockPhilox - 1 (c is a multiple of
        // kBlockPhilox, so c_lo + h never carries into c_hi)
        float rr[T][2 * kBlockPhilox], tg[T][kBlockSteps];
#pragma unroll
        for (int t = 0; t < T; ++t) {
            // the block's Philox words first, then their Box-Muller pairs (measured +0.4 % over
            // interleaving them per call: the MUFU work of the pairs comes in one stretch)
            uint4 xs[kBlockPhilox];
#pragma unroll
            for (int h = 0; h < kBlockPhilox; ++h) xs[h] = philox_lane_block(L[t].P, L[t].c_lo, static_cast<unsigned>(h));
#pragma unroll
            for (int h = 0; h < kBlockPhilox; ++h) {
                bm_pair_f32(xs[h].x, xs[h].y, L[t].bmc, rr[t][2 * h], tg[t][4 * h], tg[t][4 * h + 1]);
                bm_pair_f32(xs[h].z, xs[h].w, L[t].bmc, rr[t][2 * h + 1], tg[t][4 * h + 2], tg[t][4 * h + 3]);
            }
            if constexpr (R) bias_line(fmaf(L[t].nudt, L[t].Jf, L[t].gb), L[t].nudt, L[t].dt, gs[t], gsl[t]);
        }
        // The block's steps without a branch: each lane only tracks the largest phase of the block.
        // In the rare block where it reached the lane's bound hb, the lane's block is replayed
        // (in the warp's event path below) from the saved start state with the event test after
        // every step, so wraps and the escape step are exactly those of a step-by-step test.
        float r0s[T], v0s[T], mx[T];
#pragma unroll
        for (int t = 0; t < T; ++t) {
            r0s[t] = L[t].r;
            v0s[t] = L[t].v;
            mx[t] = -INFINITY;
        }
#pragma unroll
        for (int s = 0; s < kBlockSteps; ++s) {
#pragma unroll
            for (int t = 0; t < T; ++t) {
                step_f32<M, H>(L[t].r, L[t].v, rr[t][s >> 1], tg[t][s], bias_b0<H, R>(gs[t], gsl[t], s),
                               bias_b1<H, R>(gs[t], gsl[t], s), L[t].dt, L[t].A, L[t].amp);
                mx[t] = fmaxf(mx[t], L[t].r);
            }
        }
        bool ev = false;
#pragma unroll
        for (int t = 0; t < T; ++t) {
            L[t].c_lo += kBlockPhilox;
            if constexpr (R) L[t].Jf += static_cast<float>(kBlockSteps);
            L[t].budget -= 1u;
            // one vote covers every rare case: a bound reached (escape or upper wrap), the
            // countdown (step budget, bias re-base, low-word carry) and the lower wrap
            ev |= (mx[t] >= L[t].hb) || (L[t].budget == 0u) || (L[t].r < -kPiF);
        }
        ++b;
        if (__any_sync(kFull, ev)) {
            useful += static_cast<unsigned long long>(kBlockSteps) * static_cast<unsigned>(n_active) * (b - b_count);
            b_count = b;
#pragma unroll
            for (int t = 0; t < T; ++t) {
                if (mx[t] >= L[t].hb) {
                    L[t].r = r0s[t];
                    L[t].v = v0s[t];
#pragma unroll
                    for (int s = 0; s < kBlockSteps; ++s) {
                        step_f32<M, H>(L[t].r, L[t].v, rr[t][s >> 1], tg[t][s],
                                       bias_b0<H, R>(gs[t], gsl[t], s), bias_b1<H, R>(gs[t], gsl[t], s),
                                       L[t].dt, L[t].A, L[t].amp);
                        if (L[t].r >= L[t].hb) phase_event(L[t], E, s);
                    }
                }
                if (L[t].r < -kPiF) wrap_down(L[t], E);
                if (L[t].slot >= 0 && L[t].c_lo == 0u) {   // 2^32-block carry: new fixed words
                    L[t].c_hi += 1u;
                    const SlotDev *S = E.slots + L[t].slot;
                    philox_lane_init(L[t].P, S->key0, S->key1, L[t].c_hi, L[t].gid_lo, L[t].gid_hi);
                }
            }
            finish_lanes(L, E, V, useful, n_active, n_esc, n_cens);
            refill(L, E, V, kind_of(M, H, R), n_active, cursor, b);
            if (!__any_sync(kFull, n_active > 0)) break;
            if constexpr (!R) {
#pragma unroll
                for (int t = 0; t < T; ++t)
                    bias_line(fmaf(L[t].nudt, L[t].Jf, L[t].gb), L[t].nudt, L[t].dt, gs[t], gsl[t]);
            }
        }
    }
    useful += static_cast<unsigned long long>(kBlockSteps) * static_cast<unsigned>(n_active) * (b - b_count);
    return b;
}

// One trajectory per thread runs best as one CTA of 640 threads per SM: 20 warps, five per
// scheduler, at 96 registers (measured against 512, 576, 672 and 768); two per thread as CTAs
// of up to 256.
// An idle warp looks for work of any kind, starting from a warp-dependent one; returns the kind
// it took work of, or -1.
template <int T>
__device__ __forceinline__ int seek_work(Lane (&L)[T], const EngineDev &E, const CtaView &V, int &n_active,
                                         unsigned &cursor, unsigned b) {
    const unsigned warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int first = static_cast<int>(warp % kNumKinds);
    for (int q = 0; q < kNumKinds; ++q) {
        const int m = (first + q) % kNumKinds;
        refill(L, E, V, m, n_active, cursor, b);
        if (__any_sync(kFull, n_active > 0)) return m;
    }
    return -1;
}

template <int T>
__global__ void __launch_bounds__(T == 1 ? 640 : 256, 1) engine_chunk_kernel(EngineDev E) {
    const unsigned nthreads = gridDim.x * blockDim.x;
    const unsigned gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned warp = gtid >> 5;
    const int lane = threadIdx.x & 31;
    // This CTA's view of the requests for the launch: which listed requests have ids or suspended
    // trajectories to hand out, and how many of its lanes hold each.
    __shared__ unsigned sh_ok[kMaxRequests];
    __shared__ int sh_held[kMaxRequests], sh_budget[kMaxRequests];
    __shared__ int sh_res_slot[32], sh_res_cnt[32], sh_started[32];   // a CTA has at most 32 warps
    __shared__ unsigned long long sh_res_base[32];
    __shared__ int sh_pool;
    __shared__ unsigned sh_chunk;
    const CtaView V{sh_ok, sh_held, sh_budget, sh_res_slot, sh_res_cnt, sh_res_base, sh_started, &sh_pool};
    for (int s = threadIdx.x; s < E.max_requests; s += blockDim.x) {
        sh_ok[s] = 0u;
        sh_held[s] = 0;
        sh_budget[s] = 0;
    }
    if (threadIdx.x == 0) {
        sh_pool = 0;
        // blocks per warp of this launch: the engine's full launch or a shorter one it chose
        const unsigned c = static_cast<unsigned>(*E.chunk_now);
        sh_chunk = c == 0u || c > E.chunk_blocks ? E.chunk_blocks : c;
    }
    if (threadIdx.x < 32) {
        sh_res_slot[threadIdx.x] = -1;
        sh_res_cnt[threadIdx.x] = 0;
        sh_res_base[threadIdx.x] = 0ull;
        sh_started[threadIdx.x] = 0;
    }
    __syncthreads();
    {
        int listed = 0;
        for (int k = 0; k < kNumKinds; ++k) listed += E.act_count[k];
        for (int i = threadIdx.x; i < listed; i += blockDim.x) {
            int k = 0, j = i;
            while (j >= E.act_count[k]) j -= E.act_count[k++];
            const int s = E.act_list[k * E.max_requests + j];
            const SlotCtl &C = E.ctl[s];
            if (vload(C.state) != kSlotActive) continue;
            sh_ok[s] = (vload(C.head) < E.slots[s].n_traj ? 1u : 0u) | (vload(C.park_avail) > 0 ? 2u : 0u);
            // reservoir room: what the ring can still take beyond one entry per lane (the most
            // suspensions of this launch could add), shared equally by the CTAs
            const long long room = static_cast<long long>(E.slots[s].park_cap) - vload(C.park_used) -
                                   static_cast<long long>(E.n_lanes);
            sh_budget[s] = room > 0 ? static_cast<int>(room / gridDim.x) : 0;
        }
    }
    Lane L[T];
    int n_active = 0;
#pragma unroll
    for (int t = 0; t < T; ++t) {
        const unsigned i = t * nthreads + gtid;
        int s = checked(E, i < E.n_lanes, kChkLane) ? E.lanes.slot[i] : -1;
        if (s >= 0 && !checked(E, s < E.max_requests, kChkSlot)) s = -1;
        if (s >= 0 && vload(E.ctl[s].state) != kSlotActive) {   // request finished or cancelled
            atomicSub(&E.ctl[s].inflight, 1);
            s = -1;
        }
        if (s < 0) {
            set_idle(L[t]);
            continue;
        }
        const SlotDev *S = E.slots + s;
        L[t].slot = s;
        L[t].r = E.lanes.r[i];
        L[t].v = E.lanes.v[i];
        L[t].hb = E.lanes.hb[i];
        L[t].w = E.lanes.w[i];
        L[t].c_lo = E.lanes.c_lo[i];
        L[t].c_hi = E.lanes.c_hi[i];
        L[t].gid_lo = E.lanes.gid_lo[i];
        L[t].gid_hi = E.lanes.gid_hi[i];
        L[t].esc = -1;
        load_consts(L[t], S);
        set_progress(L[t], S);
        atomicAdd(&sh_held[s], 1);
        ++n_active;
    }
    __syncthreads();
    int kind = E.warp_kind[warp];
    if (kind >= 0 && !checked(E, kind < kNumKinds, kChkKind)) kind = -1;
    if (!__any_sync(kFull, n_active > 0)) kind = -1;
    unsigned cursor = E.warp_cursor[warp];
    unsigned long long useful = 0;
    unsigned n_esc = 0, n_cens = 0;
    unsigned b = 0;
    if (kind >= 0) refill(L, E, V, kind, n_active, cursor, 0u);
    else kind = seek_work(L, E, V, n_active, cursor, 0u);
    // The CTA's pool holds the last 1/kPoolDiv of the launch's blocks of every warp that has work
    // now, so a CTA whose warps are partly idle (fewer trajectories than lanes) gives its busy
    // warps as many blocks as a full CTA does, and all CTAs end together.
    if (lane == 0 && kind >= 0) atomicAdd(&sh_pool, static_cast<int>(sh_chunk / kPoolDiv));
    __syncthreads();
    unsigned limit = sh_chunk - sh_chunk / kPoolDiv;
    while (b < limit || grant(V, limit)) {
        if (kind < 0) {
            kind = seek_work(L, E, V, n_active, cursor, b);
            if (kind < 0) break;
        }
        switch (kind) {
#define FPT_KIND_CASE(M_, H_, R_)                                                              \
    case kind_of(M_, H_, R_):                                                                \
        b = run_blocks<M_, H_, R_, T>(L, E, V, b, n_active, cursor, useful, n_esc, n_cens, limit); \
        break;
        FPT_KIND_CASE(kUnder, kEuler, kConstBias)
        FPT_KIND_CASE(kOver, kEuler, kConstBias)
        FPT_KIND_CASE(kUnder, kHeun, kConstBias)
        FPT_KIND_CASE(kOver, kHeun, kConstBias)
        FPT_KIND_CASE(kUnder, kEuler, kRamp)
        FPT_KIND_CASE(kOver, kEuler, kRamp)
        FPT_KIND_CASE(kUnder, kHeun, kRamp)
        default:
            b = run_blocks<kOver, kHeun, kRamp, T>(L, E, V, b, n_active, cursor, useful, n_esc, n_cens, limit);
            break;
#undef FPT_KIND_CASE
        }
        if (!__any_sync(kFull, n_active > 0)) kind = -1;
    }
    // Preemption: a whole warp of this kind may be asked to vacate (so it can switch kind),
    // or single lanes of requests above their share to suspend.  Suspended state goes to the
    // request's ring; a push needs a free ring entry (park_used < park_cap).
    bool vacate = false;
    if (kind >= 0 && __any_sync(kFull, n_active > 0)) {
        int v = 0;
        if (lane == 0 && vload(E.vacate[kind]) > 0) v = atomicSub(&E.vacate[kind], 1) > 0 ? 1 : 0;
        vacate = __shfl_sync(kFull, v, 0) != 0;
    }
#pragma unroll
    for (int t = 0; t < T; ++t) {
        const int s = L[t].slot;
        if (s < 0) continue;
        bool park = vacate;
        if (!park && vload(E.preempt[s]) > 0) park = atomicSub(&E.preempt[s], 1) > 0;
        if (!park) continue;
        SlotCtl *C = E.ctl + s;
        const SlotDev *S = E.slots + s;
        if (atomicAdd(&C->park_used, 1) >= static_cast<int>(S->park_cap)) {
            atomicSub(&C->park_used, 1);
            continue;
        }
        const unsigned pi = atomicAdd(&C->park_tail, 1u);
        if (!checked(E, pi % S->park_cap < S->park_cap, kChkPark)) continue;
        ParkEntry &P = S->park[pi % S->park_cap];
        P.r = L[t].r;
        P.v = L[t].v;
        P.w = L[t].w;
        P.c_lo = L[t].c_lo;
        P.c_hi = L[t].c_hi;
        P.gid_lo = L[t].gid_lo;
        P.gid_hi = L[t].gid_hi;
        P.pad = 0;
        atomicSub(&C->inflight, 1);
        L[t].slot = -1;
        --n_active;
    }
    // Ids left in this warp's reservoir go back to their request as suspended trajectories that
    // have not started (state r0, v0, w0 at step 0: resuming one is starting it).  The CTA's
    // budget kept the ring's room for them.
    {
        __syncwarp();
        const int wl = static_cast<int>(threadIdx.x >> 5);
        const int rs = sh_res_slot[wl], rc = sh_res_cnt[wl];
        if (rs >= 0 && rc > 0 && checked(E, rs < E.max_requests, kChkSlot)) {
            SlotCtl *C = E.ctl + rs;
            const SlotDev *S = E.slots + rs;
            for (int j = lane; j < rc; j += 32) {
                const unsigned long long gid = S->traj_offset + sh_res_base[wl] + static_cast<unsigned long long>(j);
                const int used = atomicAdd(&C->park_used, 1);
                checked(E, used < static_cast<int>(S->park_cap), kChkPark);   // the budget's invariant
                const unsigned pi = atomicAdd(&C->park_tail, 1u);
                if (!checked(E, pi % S->park_cap < S->park_cap, kChkPark)) continue;
                ParkEntry &P = S->park[pi % S->park_cap];
                P.r = S->r0;
                P.v = S->v0;
                P.w = S->w0;
                P.c_lo = P.c_hi = 0u;
                P.gid_lo = static_cast<unsigned>(gid);
                P.gid_hi = static_cast<unsigned>(gid >> 32);
                P.pad = 0;
            }
        }
    }
    if (!__any_sync(kFull, n_active > 0)) kind = -1;
#pragma unroll
    for (int t = 0; t < T; ++t) {
        const unsigned i = t * nthreads + gtid;
        if (!checked(E, i < E.n_lanes, kChkLane)) continue;
        E.lanes.slot[i] = L[t].slot;
        if (L[t].slot < 0) continue;
        E.lanes.r[i] = L[t].r;
        E.lanes.v[i] = L[t].v;
        E.lanes.hb[i] = L[t].hb;
        E.lanes.w[i] = L[t].w;
        E.lanes.c_lo[i] = L[t].c_lo;
        E.lanes.c_hi[i] = L[t].c_hi;
        E.lanes.gid_lo[i] = L[t].gid_lo;
        E.lanes.gid_hi[i] = L[t].gid_hi;
    }
    if (lane == 0) {
        E.warp_kind[warp] = kind;
        E.warp_cursor[warp] = cursor;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        useful += __shfl_down_sync(kFull, useful, off);
        n_esc += __shfl_down_sync(kFull, n_esc, off);
        n_cens += __shfl_down_sync(kFull, n_cens, off);
    }
    if (lane == 0) {
        if (useful) atomicAdd(&E.counters[kCntUseful], useful);
        if (n_esc) atomicAdd(&E.counters[kCntEscapes], static_cast<unsigned long long>(n_esc));
        if (n_cens) atomicAdd(&E.counters[kCntCensored], static_cast<unsigned long long>(n_cens));
    }
}

__device__ __forceinline__ double u128_to_d(unsigned long long lo, unsigned long long hi) {
    return __dadd_rn(__dmul_rn(static_cast<double>(hi), 18446744073709551616.0),
                     static_cast<double>(lo));
}

// lo:hi (128 bits) += l0 + 2^32 l1 + 2^64 l2, exactly (l0, l1, l2 < 2^64).
__device__ __forceinline__ void add_limbs(unsigned long long &lo, unsigned long long &hi, unsigned long long l0,
                                          unsigned long long l1, unsigned long long l2) {
    const unsigned long long a = l1 << 32, ah = l1 >> 32;   // 2^32 l1 = ah:a
    lo += l0;
    hi += lo < l0 ? 1ull : 0ull;
    lo += a;
    hi += ah + (lo < a ? 1ull : 0ull) + l2;
}

// Fold completed id blocks, in id order, into each request's running sums; stop at the first
// prefix meeting the relative-standard-error rule, or when every block is complete.
__global__ void engine_scan_kernel(EngineDev E) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= E.max_requests) return;
    SlotCtl *C = E.ctl + s;
    if (C->state != kSlotActive) return;
    const SlotDev *S = E.slots + s;
    // entries suspended during the launch become available to the next launch's refills
    C->park_avail += static_cast<int>(C->park_tail - C->park_commit);
    C->park_commit = C->park_tail;
    unsigned p = C->prefix;
    bool finished = false;
    while (p < S->n_idblocks) {
        const unsigned long long first = static_cast<unsigned long long>(p) * S->stop_block;
        const unsigned long long left = S->n_traj - first;
        const unsigned need = left < S->stop_block ? static_cast<unsigned>(left) : S->stop_block;
        const IdBlockAcc &A = S->acc[p];
        if (A.done < need) break;
        C->n_done += A.done;
        C->n_esc += A.escaped;
        C->under += A.under;
        C->over += A.over;
        add_limbs(C->s1_lo, C->s1_hi, A.s1[0], A.s1[1], 0ull);
        add_limbs(C->s2_lo, C->s2_hi, A.s2[0], A.s2[1], A.s2[2]);
        ++p;
        if (S->stop_rse > 0.0 && C->n_esc >= 2) {
            const double n = static_cast<double>(C->n_esc);
            const double s1 = u128_to_d(C->s1_lo, C->s1_hi);
            const double s2 = u128_to_d(C->s2_lo, C->s2_hi);
            const double mk = __ddiv_rn(s1, n);
            double vk = __ddiv_rn(__dsub_rn(s2, __dmul_rn(s1, mk)), __dsub_rn(n, 1.0));
            if (vk < 0.0) vk = 0.0;
            const double mx = S->output == FPT_OUT_TIME ? __dmul_rn(S->out_b, mk)
                                                        : __dadd_rn(S->out_a, __dmul_rn(S->out_b, mk));
            const double se = __dmul_rn(fabs(S->out_b), __dsqrt_rn(__ddiv_rn(vk, n)));
            if (se <= __dmul_rn(S->stop_rse, fabs(mx))) {
                finished = true;
                break;
            }
        }
    }
    C->prefix = p;
    if (p >= S->n_idblocks) finished = true;
    if (finished) C->state = kSlotFinished;
}

}  // namespace

cudaError_t launch_engine_chunk(const EngineDev &E, int T, unsigned grid, unsigned block,
                                cudaStream_t s) {
    if (T == 1) engine_chunk_kernel<1><<<grid, block, 0, s>>>(E);
    else engine_chunk_kernel<2><<<grid, block, 0, s>>>(E);
    return cudaGetLastError();
}

cudaError_t launch_engine_scan(const EngineDev &E, cudaStream_t s) {
    const unsigned block = 128;
    const unsigned grid = (static_cast<unsigned>(E.max_requests) + block - 1) / block;
    engine_scan_kernel<<<grid, block, 0, s>>>(E);
    return cudaGetLastError();
}

cudaError_t engine_chunk_occupancy(int T, int block, int *blocks_per_sm) {
    if (T == 1)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, engine_chunk_kernel<1>,
                                                             block, 0);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, engine_chunk_kernel<2>,
                                                         block, 0);
}

}  // namespace fpt
