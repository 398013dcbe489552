// noalloc.cu -- fpt_run_noalloc: the lane-refill integration of one request, run to completion
// in a single launch, whose scratch lives in a fixed device array instead of memory the library
// allocates.
//
// Who needs this: callers that must not allocate device memory while they run -- for example a
// host program that reserved the device memory for its own pool before loading this library,
// code inside a latency-critical loop where cudaMalloc's implicit synchronisation is not
// acceptable, or plugin hosts whose contract forbids allocation during execution.  The
// persistent engine (fpt_create / fpt_submit) allocates its lane state and accumulators;
// this entry point allocates nothing.
//
// Scratch: kNoAllocScratchBytes (8 MiB) in a file-scope __device__ array, held by every GPU
// that loads the library until the process exits.  Layout: a 256-byte header (queue head,
// finished-CTA counter), then one record per CTA (exact partial sums + per-bin counts).  When
// the records of a full grid do not fit (many histogram bins) the launch uses fewer CTAs.
// Every call shares the array and it keeps the previous call's contents; the header is cleared
// on the stream before each launch.  Calls that overlap on the GPU race on it.
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>

#include "fpt_device.cuh"
#include "internal.h"

namespace fpt {
namespace {

constexpr size_t kNoAllocScratchBytes = 8u << 20;
constexpr size_t kHeaderBytes = 256;
constexpr int kBlock = 256;
constexpr unsigned kFullMask = 0xFFFFFFFFu;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

struct NoAllocArgs {
    int model, output, nbins;
    unsigned key0, key1;
    unsigned long long traj_offset, n_traj, max_steps, nblocks;
    float dt, A, amp, bmc, nudt, v0, r0, eb0;
    int w0;
    double gamma0, nudt_d, out_a, out_b, lo, hi, inv_w;
    long long *steps;              // optional per-trajectory output
    fpt_sums *sums;                // accumulated output
    unsigned long long *hist;      // accumulated output (nbins)
    unsigned char *scratch;        // device address of g_noalloc_scratch
    size_t rec_bytes;
};

__device__ __forceinline__ void add128(unsigned long long &lo, unsigned long long &hi,
                                       unsigned long long alo, unsigned long long ahi) {
    lo += alo;
    hi += ahi + (lo < alo ? 1ull : 0ull);
}

// Single-precision lane state (same step as the engine and the plain FP32 kernel).
struct NLane {
    float r, v, hb, gb, Jf;      // Jf = 4 x blocks since the bias base gb was set
    int w, esc;
    bool active;
    unsigned long long idx, c;   // trajectory index within the request, completed blocks
};

__device__ __forceinline__ void nl_start(NLane &L, const NoAllocArgs &a, unsigned long long idx) {
    L.active = true;
    L.idx = idx;
    L.c = 0;
    L.Jf = 0.0f;
    L.r = a.r0;
    L.v = a.v0;
    L.w = a.w0;
    L.hb = fminf(a.eb0, kPiF);
    L.esc = -1;
    L.gb = static_cast<float>(a.gamma0);
}

// Warp-aggregated claim of the next trajectory for every lane that needs one.  Once the queue
// is exhausted (warp-uniform flag) no further atomics are issued.
__device__ __forceinline__ void nl_claim(NLane &L, const NoAllocArgs &a, unsigned long long *head,
                                         bool &exhausted) {
    if (exhausted) return;
    const int lane = threadIdx.x & 31;
    const unsigned need = __ballot_sync(kFullMask, !L.active);
    if (!need) return;
    const int leader = __ffs(need) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(head, static_cast<unsigned long long>(__popc(need)));
    base = __shfl_sync(kFullMask, base, leader);
    if (base + __popc(need) >= a.n_traj) exhausted = true;
    if (!L.active) {
        const unsigned long long idx = base + __popc(need & ((1u << lane) - 1u));
        if (idx < a.n_traj) nl_start(L, a, idx);
    }
}

template <int M, int H, int R>
__global__ void __launch_bounds__(kBlock) noalloc_kernel(NoAllocArgs a) {
    extern __shared__ unsigned int sh_hist[];
    __shared__ unsigned long long sh_sums[8];   // done, escaped, s1 lo/hi, s2 lo/hi, under, over
    __shared__ bool sh_last;
    for (int b = threadIdx.x; b < a.nbins; b += blockDim.x) sh_hist[b] = 0;
    if (threadIdx.x < 8) sh_sums[threadIdx.x] = 0;
    __syncthreads();
    unsigned long long *head = reinterpret_cast<unsigned long long *>(a.scratch);
    unsigned *ctas_done = reinterpret_cast<unsigned *>(a.scratch + 8);

    NLane L;
    L.active = false;
    L.esc = -1;
    L.r = __int_as_float(0x7FFFFFFF);
    L.v = L.hb = L.gb = L.Jf = 0.0f;
    L.w = 0;
    L.idx = L.c = 0;
    bool exhausted = false;
    nl_claim(L, a, head, exhausted);
    unsigned long long done = 0, esc = 0, s1lo = 0, s1hi = 0, s2lo = 0, s2hi = 0, under = 0, over = 0;

    while (__any_sync(kFullMask, L.active)) {
        float rr[2 * kBlockPhilox], tg[kBlockSteps];
#pragma unroll
        for (int h = 0; h < kBlockPhilox; ++h) {
            const unsigned long long b = L.c + h;
            const uint4 x = philox4x32_10(
                make_uint4(static_cast<unsigned>(b), static_cast<unsigned>(b >> 32),
                           static_cast<unsigned>(a.traj_offset + L.idx),
                           static_cast<unsigned>((a.traj_offset + L.idx) >> 32)),
                a.key0, a.key1);
            bm_pair_f32(x.x, x.y, a.bmc, rr[2 * h], tg[4 * h], tg[4 * h + 1]);
            bm_pair_f32(x.z, x.w, a.bmc, rr[2 * h + 1], tg[4 * h + 2], tg[4 * h + 3]);
        }
        float gs, gsl;
        bias_line(fmaf(a.nudt, L.Jf, L.gb), a.nudt, a.dt, gs, gsl);
#pragma unroll
        for (int s = 0; s < kBlockSteps; ++s) {
            step_f32<M, H>(L.r, L.v, rr[s >> 1], tg[s], bias_b0<H, R>(gs, gsl, s),
                           bias_b1<H, R>(gs, gsl, s), a.dt, a.A, a.amp);
            if (L.r >= L.hb) {
                const float eb = fmaf(-kTwoPiF, static_cast<float>(L.w - a.w0), a.eb0);
                if (L.r >= eb) {
                    if (L.esc < 0) L.esc = s;
                    L.r = __int_as_float(0x7FFFFFFF);
                } else {
                    L.r -= kTwoPiF;
                    L.w += 1;
                    L.hb = fminf(fmaf(-kTwoPiF, static_cast<float>(L.w - a.w0), a.eb0), kPiF);
                }
            }
        }
        if (L.r < -kPiF) {   // lower wrap at the block end
            L.r += kTwoPiF;
            L.w -= 1;
            L.hb = fminf(fmaf(-kTwoPiF, static_cast<float>(L.w - a.w0), a.eb0), kPiF);
        }
        if (L.active) {
            L.c += kBlockPhilox;
            L.Jf += static_cast<float>(kBlockSteps);
            if ((L.c & ((1ull << 20) - 1)) == 0) {   // re-base the single-precision bias
                L.gb = static_cast<float>(a.gamma0 + a.nudt_d * static_cast<double>(4ull * L.c));
                L.Jf = 0.0f;
            }
            const bool out = L.c >= a.nblocks;
            if (L.esc >= 0 || out) {
                unsigned long long k = 0;
                bool escaped = false;
                if (L.esc >= 0) {
                    k = 4ull * (L.c - kBlockPhilox) + static_cast<unsigned long long>(L.esc) + 1ull;
                    escaped = k <= a.max_steps;
                }
                done += 1;
                if (escaped) {
                    esc += 1;
                    add128(s1lo, s1hi, k, 0ull);
                    add128(s2lo, s2hi, k * k, __umul64hi(k, k));
                    const double kd = static_cast<double>(k);
                    const double xv = a.output == FPT_OUT_TIME
                                          ? __dmul_rn(a.out_b, kd)
                                          : __dadd_rn(a.out_a, __dmul_rn(a.out_b, kd));
                    if (xv < a.lo) {
                        under += 1;
                    } else if (xv >= a.hi) {
                        over += 1;
                    } else {
                        int bin = static_cast<int>(floor(__dmul_rn(__dsub_rn(xv, a.lo), a.inv_w)));
                        if (bin >= a.nbins) bin = a.nbins - 1;
                        atomicAdd(&sh_hist[bin], 1u);
                    }
                }
                if (a.steps) a.steps[L.idx] = escaped ? static_cast<long long>(k) : -1ll;
                L.active = false;
                L.esc = -1;
                L.r = __int_as_float(0x7FFFFFFF);
            }
        }
        nl_claim(L, a, head, exhausted);
    }
    // CTA partials: registers -> shared -> this CTA's record in the scratch array
    atomicAdd(&sh_sums[0], done);
    atomicAdd(&sh_sums[1], esc);
    atomicAdd(&sh_sums[6], under);
    atomicAdd(&sh_sums[7], over);
    {   // 128-bit sums: add low words, carry counted separately
        const unsigned long long o1 = atomicAdd(&sh_sums[2], s1lo);
        atomicAdd(&sh_sums[3], s1hi + (o1 + s1lo < o1 ? 1ull : 0ull));
        const unsigned long long o2 = atomicAdd(&sh_sums[4], s2lo);
        atomicAdd(&sh_sums[5], s2hi + (o2 + s2lo < o2 ? 1ull : 0ull));
    }
    __syncthreads();
    unsigned char *rec = a.scratch + kHeaderBytes + static_cast<size_t>(blockIdx.x) * a.rec_bytes;
    unsigned long long *rs = reinterpret_cast<unsigned long long *>(rec);
    unsigned int *rh = reinterpret_cast<unsigned int *>(rec + 64);
    if (threadIdx.x < 8) rs[threadIdx.x] = sh_sums[threadIdx.x];
    for (int b = threadIdx.x; b < a.nbins; b += blockDim.x) rh[b] = sh_hist[b];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) sh_last = atomicAdd(ctas_done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!sh_last) return;
    // the last CTA folds every record into the caller's outputs
    __threadfence();
    for (int b = threadIdx.x; b < a.nbins; b += blockDim.x) {
        unsigned long long t = 0;
        for (unsigned g = 0; g < gridDim.x; ++g)
            t += reinterpret_cast<const volatile unsigned int *>(
                a.scratch + kHeaderBytes + static_cast<size_t>(g) * a.rec_bytes + 64)[b];
        if (t) atomicAdd(&a.hist[b], t);
    }
    if (threadIdx.x == 0) {
        unsigned long long f[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (unsigned g = 0; g < gridDim.x; ++g) {
            const volatile unsigned long long *r = reinterpret_cast<const volatile unsigned long long *>(
                a.scratch + kHeaderBytes + static_cast<size_t>(g) * a.rec_bytes);
            f[0] += r[0];
            f[1] += r[1];
            add128(f[2], f[3], r[2], r[3]);
            add128(f[4], f[5], r[4], r[5]);
            f[6] += r[6];
            f[7] += r[7];
        }
        unsigned long long *o = reinterpret_cast<unsigned long long *>(a.sums);
        atomicAdd(&o[0], f[0]);
        atomicAdd(&o[1], f[1]);
        const unsigned long long p1 = atomicAdd(&o[2], f[2]);
        atomicAdd(&o[3], f[3] + (p1 + f[2] < p1 ? 1ull : 0ull));
        const unsigned long long p2 = atomicAdd(&o[4], f[4]);
        atomicAdd(&o[5], f[5] + (p2 + f[4] < p2 ? 1ull : 0ull));
        atomicAdd(&o[6], f[6]);
        atomicAdd(&o[7], f[7]);
    }
}

// The current CUDA context's handle, through the driver entry point the runtime exposes (the
// library does not link the driver library itself); nullptr if it cannot be had.
using CtxGetCurrentFn = int (*)(void **);   // cuCtxGetCurrent(CUcontext *)
void *current_context() {
    static CtxGetCurrentFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<CtxGetCurrentFn>(p);
    });
    void *ctx = nullptr;
    if (fn && fn(&ctx) != 0) ctx = nullptr;
    return ctx;
}

// Device address of the scratch array: set up once per device, with that device current, and
// set up again if the device's context has changed since (after cudaDeviceReset the module is
// loaded anew and the array may live at another address).
std::mutex g_sym_mu;
struct SymEntry {
    void *ptr = nullptr;
    void *ctx = nullptr;
};
SymEntry g_sym[64];

fpt_status scratch_address(int dev, unsigned char **out) {
    std::lock_guard<std::mutex> lk(g_sym_mu);
    if (dev < 0 || dev >= 64) {
        set_error("device ordinal out of range for the no-alloc scratch table");
        return FPT_EINVAL;
    }
    void *ctx = current_context();
    if (!g_sym[dev].ptr || g_sym[dev].ctx != ctx) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error(std::string("cudaGetSymbolAddress(no-alloc scratch): ") + cudaGetErrorString(e));
            return FPT_ECUDA;
        }
        g_sym[dev].ptr = p;
        g_sym[dev].ctx = ctx;
    }
    *out = static_cast<unsigned char *>(g_sym[dev].ptr);
    return FPT_OK;
}

}  // namespace
}  // namespace fpt

using namespace fpt;

extern "C" fpt_status fpt_run_noalloc(const fpt_params *params, uint64_t n_traj, uint64_t seed,
                                      int64_t *d_steps, fpt_sums *d_sums, uint64_t *d_hist,
                                      void *stream) {
    Decoded d;
    std::string err;
    if (!decode(params, &d, &err)) {
        set_error(err);
        return FPT_EINVAL;
    }
    if (params->precision != FPT_FP32) {
        set_error("fpt_run_noalloc integrates in FP32 only");
        return FPT_EINVAL;
    }
    if (params->stop_rse != 0.0) {
        set_error("fpt_run_noalloc runs every trajectory: stop_rse must be 0");
        return FPT_EINVAL;
    }
    if (!d_sums || !d_hist) {
        set_error("d_sums and d_hist are required device outputs");
        return FPT_EINVAL;
    }
    if (n_traj > 0xFFFFFFFFull) {   // a CTA's per-bin counts are 32-bit
        set_error("fpt_run_noalloc: n_traj must be < 2^32");
        return FPT_EINVAL;
    }
    if (n_traj == 0) return FPT_OK;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t shmem = static_cast<size_t>(d.hist_bins) * 4;
    if (shmem > 40 * 1024) {
        set_error("fpt_run_noalloc: hist_bins must be <= 10240 (per-CTA histogram in shared memory)");
        return FPT_EINVAL;
    }
    void (*kernel)(NoAllocArgs) = nullptr;
    switch (d.kind) {
#define FPT_KIND_CASE(M_, H_, R_) \
    case kind_of(M_, H_, R_): kernel = noalloc_kernel<M_, H_, R_>; break;
    FPT_KIND_CASE(kUnder, kEuler, kConstBias)
    FPT_KIND_CASE(kOver, kEuler, kConstBias)
    FPT_KIND_CASE(kUnder, kHeun, kConstBias)
    FPT_KIND_CASE(kOver, kHeun, kConstBias)
    FPT_KIND_CASE(kUnder, kEuler, kRamp)
    FPT_KIND_CASE(kOver, kEuler, kRamp)
    FPT_KIND_CASE(kUnder, kHeun, kRamp)
#undef FPT_KIND_CASE
    default: kernel = noalloc_kernel<kOver, kHeun, kRamp>; break;
    }
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, shmem);
    if (e != cudaSuccess) {
        set_error(std::string("fpt_run_noalloc set-up: ") + cudaGetErrorString(e));
        return FPT_ECUDA;
    }
    if (per_sm < 1) {
        set_error("fpt_run_noalloc: hist_bins too large for shared memory");
        return FPT_EINVAL;
    }
    unsigned grid = static_cast<unsigned>(sms * per_sm);
    const uint64_t lanes_needed = (n_traj + kBlock - 1) / kBlock;
    if (grid > lanes_needed) grid = static_cast<unsigned>(lanes_needed);
    // one record per CTA must fit in the fixed scratch: with many bins, run fewer CTAs (the
    // lanes claim trajectories from one queue, so any grid computes the same result)
    const size_t rec = (64 + shmem + 255) / 256 * 256;
    const size_t fit = (kNoAllocScratchBytes - kHeaderBytes) / rec;
    if (fit < 1) {
        set_error("fpt_run_noalloc: hist_bins = " + std::to_string(d.hist_bins) + " needs " +
                  std::to_string(kHeaderBytes + rec) + " bytes of scratch for one CTA, the fixed "
                  "scratch holds " + std::to_string(kNoAllocScratchBytes));
        return FPT_EINVAL;
    }
    if (grid > fit) grid = static_cast<unsigned>(fit);
    unsigned char *scratch = nullptr;
    const fpt_status st = scratch_address(dev, &scratch);
    if (st != FPT_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    e = cudaMemsetAsync(scratch, 0, kHeaderBytes, s);   // queue head and CTA counter start at 0
    if (e != cudaSuccess) {
        set_error(std::string("fpt_run_noalloc clear: ") + cudaGetErrorString(e));
        return FPT_ECUDA;
    }
    NoAllocArgs a;
    std::memset(&a, 0, sizeof(a));
    a.model = d.model;
    a.output = d.output;
    a.nbins = d.hist_bins;
    a.key0 = static_cast<unsigned>(seed);
    a.key1 = static_cast<unsigned>(seed >> 32);
    a.traj_offset = params->traj_offset;
    a.n_traj = n_traj;
    a.max_steps = d.max_steps;
    a.nblocks = (d.max_steps + 3) / 4;
    a.dt = d.dt_f;
    a.A = d.A_f;
    a.amp = d.amp_f;
    a.bmc = d.bmc_f;
    a.nudt = d.nudt_f;
    a.v0 = d.v0_f;
    a.r0 = d.r0_f;
    a.eb0 = d.eb0_f;
    a.w0 = d.w0;
    a.gamma0 = d.gamma0;
    a.nudt_d = d.nudt;
    a.out_a = d.out_a;
    a.out_b = d.out_b;
    a.lo = d.hist_lo;
    a.hi = d.hist_hi;
    a.inv_w = d.hist_inv_w;
    a.steps = reinterpret_cast<long long *>(d_steps);
    a.sums = d_sums;
    a.hist = reinterpret_cast<unsigned long long *>(d_hist);
    a.scratch = scratch;
    a.rec_bytes = rec;
    kernel<<<grid, kBlock, shmem, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("fpt_run_noalloc launch: ") + cudaGetErrorString(e));
        return FPT_ECUDA;
    }
    return FPT_OK;
}
