// plain.cu -- one trajectory per thread (the kernel structure of Alg. 1 / Alg. 3), the exact
// reduction of escape steps into sums and histograms, and random-number hooks.
//
// FP64 kernel: the arithmetic of every step is spelled out with round-to-nearest intrinsics
// (__dadd_rn, __dmul_rn, ...) so that no multiply-add is fused, in the operation order of the
// algorithm as written:
//   gamma_k = gamma0 + (nu dt) k
//   underdamped  phi_k = phi + v dt ;  v_k = (v + ((-alpha v - A sin phi) + gamma_k) dt) + sigma z
//   overdamped   phi_k = (phi + (gamma_k - A sin phi) dt) + sigma z
// and for the stochastic Heun integrator (gamma_{k-1}, gamma_k at the two ends of the step)
//   underdamped  a0 = ((-alpha v) - A sin phi) + gamma_{k-1};  p = phi + v dt;
//                q = (v + a0 dt) + sigma z;  a1 = ((-alpha q) - A sin p) + gamma_k
//                phi_k = phi + ((v + q) 0.5) dt;  v_k = (v + ((a0 + a1) 0.5) dt) + sigma z
//   overdamped   f0 = gamma_{k-1} - A sin phi;  p = (phi + f0 dt) + sigma z;  f1 = gamma_k - A sin p
//                phi_k = (phi + ((f0 + f1) 0.5) dt) + sigma z
// with an unwrapped phase.  FP32 kernel: the engine's single-precision step on a wrapped phase.
#include <cstdint>
#include <cstring>
#include <string>

#include "fpt_device.cuh"
#include "internal.h"

namespace fpt {

namespace {

__device__ __forceinline__ uint32_t lo32(uint64_t x) { return static_cast<uint32_t>(x); }
__device__ __forceinline__ uint32_t hi32(uint64_t x) { return static_cast<uint32_t>(x >> 32); }

template <int M, int H>
__global__ void __launch_bounds__(128) plain_f64_kernel(PlainArgs a) {
    const uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const uint64_t gid = a.traj0 + i;
    double phi = a.phi0, v = a.v0;
    uint64_t k = 0;
    int64_t result = -1;
    for (uint64_t blk = 0; k < a.max_steps; ++blk) {
        const uint4 x = philox4x32_10(make_uint4(lo32(blk), hi32(blk), lo32(gid), hi32(gid)),
                                      a.key0, a.key1);
        double z[4];
        bm_pair_f64(x.x, x.y, z[0], z[1]);
        bm_pair_f64(x.z, x.w, z[2], z[3]);
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            if (k >= a.max_steps) break;
            k += 1;
            const double g = __dadd_rn(a.gamma0, __dmul_rn(a.nudt, static_cast<double>(k)));
            const double sn = sin(phi);
            if constexpr (H == kHeun) {
                const double g0 = __dadd_rn(a.gamma0, __dmul_rn(a.nudt, static_cast<double>(k - 1)));
                const double nz = __dmul_rn(a.sigma, z[s]);
                if constexpr (M == kUnder) {
                    const double a0 = __dadd_rn(__dsub_rn(__dmul_rn(-a.alpha, v), __dmul_rn(a.amp, sn)), g0);
                    const double p = __dadd_rn(phi, __dmul_rn(v, a.dt));
                    const double q = __dadd_rn(__dadd_rn(v, __dmul_rn(a0, a.dt)), nz);
                    const double a1 = __dadd_rn(__dsub_rn(__dmul_rn(-a.alpha, q), __dmul_rn(a.amp, sin(p))), g);
                    phi = __dadd_rn(phi, __dmul_rn(__dmul_rn(__dadd_rn(v, q), 0.5), a.dt));
                    v = __dadd_rn(__dadd_rn(v, __dmul_rn(__dmul_rn(__dadd_rn(a0, a1), 0.5), a.dt)), nz);
                } else {
                    const double f0 = __dsub_rn(g0, __dmul_rn(a.amp, sn));
                    const double p = __dadd_rn(__dadd_rn(phi, __dmul_rn(f0, a.dt)), nz);
                    const double f1 = __dsub_rn(g, __dmul_rn(a.amp, sin(p)));
                    phi = __dadd_rn(__dadd_rn(phi, __dmul_rn(__dmul_rn(__dadd_rn(f0, f1), 0.5), a.dt)), nz);
                }
            } else if constexpr (M == kUnder) {
                const double phin = __dadd_rn(phi, __dmul_rn(v, a.dt));
                const double acc = __dadd_rn(__dsub_rn(__dmul_rn(-a.alpha, v), __dmul_rn(a.amp, sn)), g);
                v = __dadd_rn(__dadd_rn(v, __dmul_rn(acc, a.dt)), __dmul_rn(a.sigma, z[s]));
                phi = phin;
            } else {
                phi = __dadd_rn(__dadd_rn(phi, __dmul_rn(__dsub_rn(g, __dmul_rn(a.amp, sn)), a.dt)),
                                __dmul_rn(a.sigma, z[s]));
            }
            if (phi >= a.th) {
                result = static_cast<int64_t>(k);
                goto done;
            }
        }
    }
done:
    a.steps[i] = result;
}

// FP32: wrapped phase r in [-pi, pi) with winding w; escape when r >= eb = phi* - 2 pi w, the
// threshold in the current cell's coordinates; hb = min(eb, pi) is the one bound tested every
// step; the lower wrap at -pi is applied at the ends of blocks of kBlockSteps steps, as in the
// engine.
template <int M, int H, int R>
__global__ void __launch_bounds__(256) plain_f32_kernel(PlainArgs a) {
    const uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const uint64_t gid = a.traj0 + i;
    float r = a.r0_f, v = a.v0_f;
    int w = a.w0;
    float hb = fminf(a.eb0_f, kPiF);
    const uint64_t nblocks = (a.max_steps + 3) / 4;
    int64_t result = -1;
    uint64_t blk = 0;
    while (blk < nblocks) {
        // re-base the single-precision bias every 2^20 blocks of the trajectory:
        // gamma_k = (gb + nudt Jf) + nudt (s + 1), Jf = 4 x blocks since the base
        const uint64_t seg_end = blk + (1ull << 20) < nblocks ? blk + (1ull << 20) : nblocks;
        const float gb = static_cast<float>(a.gamma0 + a.nudt * static_cast<double>(4 * blk));
        float Jf = 0.0f;
        for (; blk < seg_end; blk += kBlockPhilox) {
            float rr[2 * kBlockPhilox], tg[kBlockSteps];
#pragma unroll
            for (int h = 0; h < kBlockPhilox; ++h) {
                const uint64_t b = blk + h;
                const uint4 x = philox4x32_10(make_uint4(lo32(b), hi32(b), lo32(gid), hi32(gid)),
                                              a.key0, a.key1);
                bm_pair_f32(x.x, x.y, a.bmc_f, rr[2 * h], tg[4 * h], tg[4 * h + 1]);
                bm_pair_f32(x.z, x.w, a.bmc_f, rr[2 * h + 1], tg[4 * h + 2], tg[4 * h + 3]);
            }
            float gs, gsl;
            bias_line(fmaf(a.nudt_f, Jf, gb), a.nudt_f, a.dt_f, gs, gsl);
#pragma unroll
            for (int s = 0; s < kBlockSteps; ++s) {
                step_f32<M, H>(r, v, rr[s >> 1], tg[s], bias_b0<H, R>(gs, gsl, s),
                               bias_b1<H, R>(gs, gsl, s), a.dt_f, a.A_f, a.amp_f);
                if (r >= hb) {
                    // threshold in the current cell: eb = phi* - 2 pi w (same rounding as the engine)
                    const float eb = fmaf(-kTwoPiF, static_cast<float>(w - a.w0), a.eb0_f);
                    if (r >= eb) {
                        const uint64_t k = 4 * blk + s + 1;
                        if (k <= a.max_steps) result = static_cast<int64_t>(k);
                        goto done;
                    }
                    r -= kTwoPiF;
                    w += 1;
                    hb = fminf(fmaf(-kTwoPiF, static_cast<float>(w - a.w0), a.eb0_f), kPiF);
                }
            }
            if (r < -kPiF) {   // lower wrap at the block end, as in the engine
                r += kTwoPiF;
                w -= 1;
                hb = fminf(fmaf(-kTwoPiF, static_cast<float>(w - a.w0), a.eb0_f), kPiF);
            }
            Jf += static_cast<float>(kBlockSteps);
        }
    }
done:
    a.steps[i] = result;
}

__device__ __forceinline__ void add128(uint64_t &lo, uint64_t &hi, uint64_t alo, uint64_t ahi) {
    lo += alo;
    hi += ahi + (lo < alo ? 1 : 0);
}

__device__ __forceinline__ void atomic_add128(uint64_t *lo_p, uint64_t *hi_p, uint64_t alo,
                                              uint64_t ahi) {
    unsigned long long *lp = reinterpret_cast<unsigned long long *>(lo_p);
    const unsigned long long old = atomicAdd(lp, static_cast<unsigned long long>(alo));
    const uint64_t carry = (old + alo < old) ? 1 : 0;
    if (ahi + carry) atomicAdd(reinterpret_cast<unsigned long long *>(hi_p),
                               static_cast<unsigned long long>(ahi + carry));
}

constexpr int kSharedBins = 8192;

__global__ void __launch_bounds__(256) reduce_kernel(ReduceArgs a) {
    extern __shared__ unsigned int sh_hist[];
    const bool sh = a.hist && a.nbins <= kSharedBins;
    if (sh)
        for (int b = threadIdx.x; b < a.nbins; b += blockDim.x) sh_hist[b] = 0;
    __syncthreads();
    uint64_t done = 0, esc = 0, s1lo = 0, s1hi = 0, s2lo = 0, s2hi = 0, under = 0, over = 0;
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < a.n;
         i += stride) {
        const int64_t k = a.steps[i];
        done += 1;
        if (k < 0) continue;
        const uint64_t uk = static_cast<uint64_t>(k);
        esc += 1;
        add128(s1lo, s1hi, uk, 0);
        add128(s2lo, s2hi, uk * uk, __umul64hi(uk, uk));
        if (!a.hist) continue;
        const double x = a.output == FPT_OUT_TIME
                             ? __dmul_rn(a.out_b, static_cast<double>(uk))
                             : __dadd_rn(a.out_a, __dmul_rn(a.out_b, static_cast<double>(uk)));
        if (x < a.lo) {
            under += 1;
        } else if (x >= a.hi) {
            over += 1;
        } else {
            int b = static_cast<int>(floor(__dmul_rn(__dsub_rn(x, a.lo), a.inv_w)));
            if (b >= a.nbins) b = a.nbins - 1;
            if (sh) atomicAdd(&sh_hist[b], 1u);
            else atomicAdd(&a.hist[b], 1ull);
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        done += __shfl_down_sync(0xFFFFFFFFu, done, off);
        esc += __shfl_down_sync(0xFFFFFFFFu, esc, off);
        under += __shfl_down_sync(0xFFFFFFFFu, under, off);
        over += __shfl_down_sync(0xFFFFFFFFu, over, off);
        const uint64_t a1 = __shfl_down_sync(0xFFFFFFFFu, s1lo, off);
        const uint64_t b1 = __shfl_down_sync(0xFFFFFFFFu, s1hi, off);
        const uint64_t a2 = __shfl_down_sync(0xFFFFFFFFu, s2lo, off);
        const uint64_t b2 = __shfl_down_sync(0xFFFFFFFFu, s2hi, off);
        add128(s1lo, s1hi, a1, b1);
        add128(s2lo, s2hi, a2, b2);
    }
    if ((threadIdx.x & 31) == 0 && done) {
        atomicAdd(reinterpret_cast<unsigned long long *>(&a.sums->n_done), done);
        if (esc) atomicAdd(reinterpret_cast<unsigned long long *>(&a.sums->n_escaped), esc);
        if (under) atomicAdd(reinterpret_cast<unsigned long long *>(&a.sums->under), under);
        if (over) atomicAdd(reinterpret_cast<unsigned long long *>(&a.sums->over), over);
        atomic_add128(&a.sums->s1_lo, &a.sums->s1_hi, s1lo, s1hi);
        atomic_add128(&a.sums->s2_lo, &a.sums->s2_hi, s2lo, s2hi);
    }
    if (sh) {
        __syncthreads();
        for (int b = threadIdx.x; b < a.nbins; b += blockDim.x)
            if (sh_hist[b]) atomicAdd(&a.hist[b], static_cast<unsigned long long>(sh_hist[b]));
    }
}

__global__ void philox_fill_kernel(uint32_t k0, uint32_t k1, uint64_t traj, uint64_t block0,
                                   uint64_t nblocks, uint32_t *out) {
    const uint64_t j = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= nblocks) return;
    const uint64_t b = block0 + j;
    const uint4 x = philox4x32_10(make_uint4(lo32(b), hi32(b), lo32(traj), hi32(traj)), k0, k1);
    out[4 * j + 0] = x.x;
    out[4 * j + 1] = x.y;
    out[4 * j + 2] = x.z;
    out[4 * j + 3] = x.w;
}

__global__ void normals_fill_kernel(int precision, uint32_t k0, uint32_t k1, uint64_t traj,
                                    uint64_t n0, uint64_t n, double *out) {
    const uint64_t j = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const uint64_t idx = n0 + j, b = idx / 4;
    const int slot = static_cast<int>(idx % 4);
    const uint4 x = philox4x32_10(make_uint4(lo32(b), hi32(b), lo32(traj), hi32(traj)), k0, k1);
    const uint32_t w0 = slot < 2 ? x.x : x.z, w1 = slot < 2 ? x.y : x.w;
    if (precision == FPT_FP64) {
        double z0, z1;
        bm_pair_f64(w0, w1, z0, z1);
        out[j] = (slot & 1) ? z1 : z0;
    } else {
        float rr, cs, sn;
        bm_pair_f32(w0, w1, -1.3862943611198906f /* -2 ln 2: unit variance */, rr, cs, sn);
        out[j] = static_cast<double>(__fmul_rn(rr, (slot & 1) ? sn : cs));
    }
}

unsigned grid_for(uint64_t n, unsigned block) {
    return static_cast<unsigned>((n + block - 1) / block);
}

}  // namespace

cudaError_t launch_plain_f64(const PlainArgs &a, cudaStream_t s) {
    const unsigned block = 128;
    const unsigned grid = grid_for(a.n, block);
    switch (a.model + 2 * a.integrator) {
    case kUnder: plain_f64_kernel<kUnder, kEuler><<<grid, block, 0, s>>>(a); break;
    case kOver: plain_f64_kernel<kOver, kEuler><<<grid, block, 0, s>>>(a); break;
    case kUnder + 2: plain_f64_kernel<kUnder, kHeun><<<grid, block, 0, s>>>(a); break;
    default: plain_f64_kernel<kOver, kHeun><<<grid, block, 0, s>>>(a); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_plain_f32(const PlainArgs &a, cudaStream_t s) {
    const unsigned block = 256;
    const unsigned grid = grid_for(a.n, block);
    switch (a.kind) {
#define FPT_KIND_CASE(M_, H_, R_) \
    case kind_of(M_, H_, R_): plain_f32_kernel<M_, H_, R_><<<grid, block, 0, s>>>(a); break;
    FPT_KIND_CASE(kUnder, kEuler, kConstBias)
    FPT_KIND_CASE(kOver, kEuler, kConstBias)
    FPT_KIND_CASE(kUnder, kHeun, kConstBias)
    FPT_KIND_CASE(kOver, kHeun, kConstBias)
    FPT_KIND_CASE(kUnder, kEuler, kRamp)
    FPT_KIND_CASE(kOver, kEuler, kRamp)
    FPT_KIND_CASE(kUnder, kHeun, kRamp)
#undef FPT_KIND_CASE
    default: plain_f32_kernel<kOver, kHeun, kRamp><<<grid, block, 0, s>>>(a); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_reduce(const ReduceArgs &a, cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned block = 256;
    uint64_t g = (a.n + block - 1) / block;
    const uint64_t gmax = static_cast<uint64_t>(sms > 0 ? sms : 1) * 4;
    if (g > gmax) g = gmax;
    if (g == 0) g = 1;
    const size_t shmem = (a.hist && a.nbins <= kSharedBins) ? a.nbins * sizeof(unsigned int) : 0;
    reduce_kernel<<<static_cast<unsigned>(g), block, shmem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_philox_fill(uint64_t seed, uint64_t traj, uint64_t block0, uint64_t nblocks,
                               uint32_t *out, cudaStream_t s) {
    philox_fill_kernel<<<grid_for(nblocks, 256), 256, 0, s>>>(
        static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32), traj, block0, nblocks, out);
    return cudaGetLastError();
}

cudaError_t launch_normals_fill(int precision, uint64_t seed, uint64_t traj, uint64_t n0,
                                uint64_t n, double *out, cudaStream_t s) {
    normals_fill_kernel<<<grid_for(n, 256), 256, 0, s>>>(
        precision, static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32), traj, n0, n, out);
    return cudaGetLastError();
}

}  // namespace fpt

using namespace fpt;

static fpt_status cuda_fail(cudaError_t e, const char *what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return FPT_ECUDA;
}

extern "C" fpt_status fpt_plain_launch(const fpt_params *params, uint64_t seed, uint64_t traj0,
                                       uint64_t n, int64_t *d_steps, void *stream) {
    Decoded d;
    std::string err;
    if (!decode(params, &d, &err)) {
        set_error(err);
        return FPT_EINVAL;
    }
    if (params->precision != FPT_FP32 && params->precision != FPT_FP64) {
        set_error("unknown precision");
        return FPT_EINVAL;
    }
    if (n > (1ull << 32)) {
        set_error("n must be <= 2^32");
        return FPT_EINVAL;
    }
    if (n == 0) return FPT_OK;
    if (!d_steps) {
        set_error("d_steps is NULL");
        return FPT_EINVAL;
    }
    PlainArgs a;
    std::memset(&a, 0, sizeof(a));
    a.model = d.model;
    a.integrator = d.integrator;
    a.kind = d.kind;
    a.key0 = static_cast<uint32_t>(seed);
    a.key1 = static_cast<uint32_t>(seed >> 32);
    a.traj0 = traj0;
    a.n = n;
    a.steps = d_steps;
    a.max_steps = d.max_steps;
    a.alpha = d.alpha;
    a.amp = d.amp;
    a.dt = d.dt;
    a.sigma = d.sigma;
    a.gamma0 = d.gamma0;
    a.nudt = d.nudt;
    a.phi0 = d.phi0;
    a.v0 = d.v0;
    a.th = d.th;
    a.dt_f = d.dt_f;
    a.A_f = d.A_f;
    a.amp_f = d.amp_f;
    a.bmc_f = d.bmc_f;
    a.nudt_f = d.nudt_f;
    a.v0_f = d.v0_f;
    a.r0_f = d.r0_f;
    a.eb0_f = d.eb0_f;
    a.w0 = d.w0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const cudaError_t e =
        params->precision == FPT_FP64 ? launch_plain_f64(a, s) : launch_plain_f32(a, s);
    if (e != cudaSuccess) return cuda_fail(e, "plain kernel launch");
    return FPT_OK;
}

extern "C" fpt_status fpt_reduce_steps(const fpt_params *params, const int64_t *d_steps,
                                       uint64_t n, fpt_sums *d_sums, uint64_t *d_hist,
                                       void *stream) {
    Decoded d;
    std::string err;
    if (!decode(params, &d, &err)) {
        set_error(err);
        return FPT_EINVAL;
    }
    if (!d_sums || (n && !d_steps)) {
        set_error("NULL device pointer");
        return FPT_EINVAL;
    }
    if (n == 0) return FPT_OK;
    ReduceArgs a;
    a.steps = d_steps;
    a.n = n;
    a.output = d.output;
    a.out_a = d.out_a;
    a.out_b = d.out_b;
    a.lo = d.hist_lo;
    a.hi = d.hist_hi;
    a.inv_w = d.hist_inv_w;
    a.nbins = d.hist_bins;
    a.sums = d_sums;
    a.hist = reinterpret_cast<unsigned long long *>(d_hist);
    const cudaError_t e = launch_reduce(a, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "reduce kernel launch");
    return FPT_OK;
}

extern "C" fpt_status fpt_philox_fill(uint64_t seed, uint64_t traj, uint64_t block0,
                                      uint64_t nblocks, uint32_t *d_out, void *stream) {
    if (nblocks == 0) return FPT_OK;
    if (!d_out || nblocks > (1ull << 31)) {
        set_error("bad output buffer or size");
        return FPT_EINVAL;
    }
    const cudaError_t e =
        launch_philox_fill(seed, traj, block0, nblocks, d_out, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "philox fill");
    return FPT_OK;
}

extern "C" fpt_status fpt_normals_fill(int precision, uint64_t seed, uint64_t traj, uint64_t n0,
                                       uint64_t n, double *d_out, void *stream) {
    if (n == 0) return FPT_OK;
    if (!d_out || n > (1ull << 31) || (precision != FPT_FP32 && precision != FPT_FP64)) {
        set_error("bad output buffer, size or precision");
        return FPT_EINVAL;
    }
    const cudaError_t e = launch_normals_fill(precision, seed, traj, n0, n, d_out,
                                              static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "normals fill");
    return FPT_OK;
}
