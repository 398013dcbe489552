// internal.h -- host-side request decoding and shared declarations (not part of the ABI).
#pragma once

#include <cmath>
#include <cstdint>
#include <string>

#include <cuda_runtime.h>

#include "fpt.h"

namespace fpt {

// Thread-local error text for entry points without an engine.
void set_error(const std::string &msg);
const std::string &get_error();

constexpr uint64_t kMaxSteps = 1ull << 48;
// Steps per block of the single-precision kernels: kBlockPhilox Philox calls (4 normals each).
// A block runs without a branch; the escape test, the lower wrap and the bias re-base act at
// block granularity (with exact replay of a block in which a bound was reached), so every FP32
// kernel must use the same block length to agree bit for bit.
constexpr int kBlockPhilox = 4;
constexpr int kBlockSteps = 4 * kBlockPhilox;
constexpr int kMaxBins = 1 << 20;

// A request decoded on the host (the set-up of Alg. 1 / Alg. 3): double constants used
// by the FP64 kernels and by the result arithmetic, and rounded single-precision constants
// for the FP32 step.  Double quantities are evaluated in the order
//   sigma = sqrt(((2 alpha) D) dt)  (underdamped)   sigma = sqrt((2 D) dt)  (overdamped)
//   nudt = nu dt,  phi0 = asin(gamma0) when not given,  phi* = phi0 + threshold or threshold.
struct Decoded {
    int model = 0, output = 0;
    int integrator = 0;  // FPT_EULER_MARUYAMA | FPT_HEUN
    int kind = 0;        // model + 2 integrator + 4 ramp (nudt_f != 0): the FP32 code path
    double alpha = 0, D = 0, gamma0 = 0, nudt = 0, amp = 1, dt = 0, sigma = 0;
    double phi0 = 0, v0 = 0, th = 0;
    uint64_t max_steps = 0;
    // observable x = out_a + out_b * k (time: a = 0, b = dt; bias: a = gamma0, b = nu dt)
    double out_a = 0, out_b = 0;
    int hist_bins = 1;
    double hist_lo = 0, hist_hi = 1, hist_inv_w = 1;
    // single-precision step constants and the wrapped start / threshold; A_f is the underdamped
    // velocity coefficient, 1 - alpha dt for Euler and -alpha for Heun
    float dt_f = 0, A_f = 0, amp_f = 0, bmc_f = 0, nudt_f = 0, v0_f = 0;
    float r0_f = 0;      // start phase wrapped to [-pi, pi)
    int32_t w0 = 0;      // windings of the start phase
    float eb0_f = 0;     // threshold in the start cell's coordinates: phi* - 2 pi w0
};

bool decode(const fpt_params *p, Decoded *d, std::string *err);

// Observable, mean/variance and histogram bin of an escape step, in IEEE double with every
// operation rounded separately (the host compiler runs with contraction off).
inline double observable(const Decoded &d, uint64_t k) {
    if (d.output == FPT_OUT_TIME) return d.out_b * static_cast<double>(k);
    return d.out_a + d.out_b * static_cast<double>(k);
}

void sums_to_result(const Decoded &d, const fpt_sums &s, fpt_result *out);

// ---- kernels (launch wrappers; definitions in plain.cu / engine_kernels.cu) ----
struct PlainArgs {
    int model, integrator, kind;
    uint32_t key0, key1;
    uint64_t traj0, n;
    int64_t *steps;
    uint64_t max_steps;
    // FP64
    double alpha, amp, dt, sigma, gamma0, nudt, phi0, v0, th;
    // FP32
    float dt_f, A_f, amp_f, bmc_f, nudt_f, v0_f, r0_f, eb0_f;
    int32_t w0;
};
cudaError_t launch_plain_f64(const PlainArgs &a, cudaStream_t s);
cudaError_t launch_plain_f32(const PlainArgs &a, cudaStream_t s);

struct ReduceArgs {
    const int64_t *steps;
    uint64_t n;
    int output;
    double out_a, out_b, lo, hi, inv_w;
    int nbins;
    fpt_sums *sums;
    unsigned long long *hist;
};
cudaError_t launch_reduce(const ReduceArgs &a, cudaStream_t s);

cudaError_t launch_philox_fill(uint64_t seed, uint64_t traj, uint64_t block0, uint64_t nblocks,
                               uint32_t *out, cudaStream_t s);
cudaError_t launch_normals_fill(int precision, uint64_t seed, uint64_t traj, uint64_t n0,
                                uint64_t n, double *out, cudaStream_t s);

}  // namespace fpt
