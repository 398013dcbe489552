// fpt_device.cuh -- device primitives of the FPT hot path (sm_103a).
//
//   philox4x32_10   counter-based generator (Salmon et al., SC'11), all in registers
//   PhiloxLane      the same generator with the words of rounds 0-2 that no block changes kept per lane
//   bm_pair_f32     Box-Muller (Sec. III.B, nrand) in single precision, noise-scaled
//   bm_pair_f64     Box-Muller in double precision, same arithmetic order as the FP64 oracle
//   step_f32<M,H>   one Euler-Maruyama step of Alg. 1 / Alg. 3 (H = 0) or one stochastic Heun
//                   step (H = 1) on a wrapped phase
//
// Keying (fixed once for the whole library): key = (seed lo, seed hi), counter =
// (block lo, block hi, trajectory lo, trajectory hi); block b feeds steps 4b+1 .. 4b+4, words
// (x0,x1) -> normals of steps 4b+1, 4b+2 and (x2,x3) -> steps 4b+3, 4b+4.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace fpt {

constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

constexpr float kPiF = 3.14159265358979323846f;

constexpr float kTwoPiF = 6.28318530717958647692f;

// Philox4x32-10 of one trajectory, prepared for the many blocks it draws.  Counter words
// (c0, c1, c2, c3) = (block lo, block hi, trajectory lo, trajectory hi), key (k0, k1); round r
// uses the key (k0 + r W0, k1 + r W1) and maps (x, y, z, w) to
// (hi(M1 z) ^ y ^ k0r, lo(M1 z), hi(M0 x) ^ w ^ k1r, lo(M0 x)).  Only c0 changes from block to
// block (c1 only on a carry of 2^32 blocks), so for every block of the trajectory:
//   round 0: x1 = hi(M1 c2) ^ c1 ^ k0 and y1 = lo(M1 c2) are fixed; z1 = hi(M0 c0) ^ (c3 ^ k1)
//            takes a fixed mask;
//   round 1: its product M0 x1 is fixed, so z2 = hi(M0 x1) ^ w1 ^ (k1 + W1) and w2 = lo(M0 x1)
//            take fixed words, as does x2 = hi(M1 z1) ^ (y1 ^ (k0 + W0));
//   round 2: z3 = hi(M0 x2) ^ (w2 ^ (k1 + 2 W1)), with w2 fixed.
// Those fixed words, with their round keys folded in, are kept per lane with the round keys of
// rounds 2..9 (k0) and 3..9 (k1): a call costs one wide multiply in round 0 and one in round 1.
// Same output as philox4x32_10.
struct PhiloxLane {
    uint32_t ka[8];   // k0 + r W0, rounds 2..9
    uint32_t kb[7];   // k1 + r W1, rounds 3..9
    uint32_t m0;      // round 0: c3 ^ k1
    uint32_t x1m;     // round 1: y1 ^ (k0 + W0)
    uint32_t z1m;     // round 1: hi(M0 x1) ^ (k1 + W1)
    uint32_t z2m;     // round 2: lo(M0 x1) ^ (k1 + 2 W1)
};

__host__ __device__ __forceinline__ void philox_lane_init(PhiloxLane &P, uint32_t k0, uint32_t k1,
                                                          uint32_t c_hi, uint32_t t_lo, uint32_t t_hi) {
#pragma unroll
    for (int r = 2; r < 10; ++r) P.ka[r - 2] = k0 + static_cast<uint32_t>(r) * kPhiloxW0;
#pragma unroll
    for (int r = 3; r < 10; ++r) P.kb[r - 3] = k1 + static_cast<uint32_t>(r) * kPhiloxW1;
    const uint64_t p1 = static_cast<uint64_t>(kPhiloxM1) * t_lo;
    const uint32_t x1 = static_cast<uint32_t>(p1 >> 32) ^ c_hi ^ k0;
    const uint32_t y1 = static_cast<uint32_t>(p1);
    const uint64_t q0 = static_cast<uint64_t>(kPhiloxM0) * x1;          // round 1's fixed product
    P.m0 = t_hi ^ k1;
    P.x1m = y1 ^ (k0 + kPhiloxW0);
    P.z1m = static_cast<uint32_t>(q0 >> 32) ^ (k1 + kPhiloxW1);
    P.z2m = static_cast<uint32_t>(q0) ^ (k1 + 2u * kPhiloxW1);
}

// Words of block c_lo + h for h < 4 with c_lo a multiple of 4 (no carry into the high word):
// round 0's product M0 (c_lo + h) is formed as the wide multiply-add M0 c_lo + M0 h.
__host__ __device__ __forceinline__ uint4 philox_lane_block(const PhiloxLane &P, uint32_t c_lo, uint32_t h) {
    const uint64_t p0 = static_cast<uint64_t>(kPhiloxM0) * c_lo + static_cast<uint64_t>(kPhiloxM0) * h;
    const uint32_t z1 = static_cast<uint32_t>(p0 >> 32) ^ P.m0, w1 = static_cast<uint32_t>(p0);
    // round 1 (x1, y1 and the product M0 x1 are in the masks)
    const uint64_t q1 = static_cast<uint64_t>(kPhiloxM1) * z1;
    const uint32_t x2 = static_cast<uint32_t>(q1 >> 32) ^ P.x1m, y2 = static_cast<uint32_t>(q1);
    const uint32_t z2 = P.z1m ^ w1;
    // round 2 (w2 is in the mask z2m)
    const uint64_t r0 = static_cast<uint64_t>(kPhiloxM0) * x2;
    const uint64_t r1 = static_cast<uint64_t>(kPhiloxM1) * z2;
    uint4 c = make_uint4(static_cast<uint32_t>(r1 >> 32) ^ y2 ^ P.ka[0], static_cast<uint32_t>(r1),
                         static_cast<uint32_t>(r0 >> 32) ^ P.z2m, static_cast<uint32_t>(r0));
#pragma unroll
    for (int round = 3; round < 10; ++round) {
        const uint64_t a0 = static_cast<uint64_t>(kPhiloxM0) * c.x;
        const uint64_t a1 = static_cast<uint64_t>(kPhiloxM1) * c.z;
        c = make_uint4(static_cast<uint32_t>(a1 >> 32) ^ c.y ^ P.ka[round - 2], static_cast<uint32_t>(a1),
                       static_cast<uint32_t>(a0 >> 32) ^ c.w ^ P.kb[round - 3], static_cast<uint32_t>(a0));
    }
    return c;
}

// Philox4x32-10: ten rounds of two 32x32->64 multiplies; the key advances by the Weyl
// constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint64_t p0 = static_cast<uint64_t>(kPhiloxM0) * c.x;
        const uint64_t p1 = static_cast<uint64_t>(kPhiloxM1) * c.z;
        const uint32_t hi0 = static_cast<uint32_t>(p0 >> 32), lo0 = static_cast<uint32_t>(p0);
        const uint32_t hi1 = static_cast<uint32_t>(p1 >> 32), lo1 = static_cast<uint32_t>(p1);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
    return c;
}

// 1 + m 2^-23 with m = x >> 9, the high 23 bits of a word, as a float in [1, 2): one funnel
// shift of (0x7F : x) by 9 places the exponent bits of 1.0 above m.
__device__ __forceinline__ float mant_f32(uint32_t x) {
    return __uint_as_float(__funnelshift_r(x, 0x7Fu, 9));
}

// Single-precision uniform in (0, 1): u = (m + 1/2) 2^-23, the double-precision uniform
// (x + 1/2) 2^-32 rounded to 23 bits, so the FP32 and FP64 normals of one trajectory stay close.
// (1 + m 2^-23) - (1 - 2^-24) is exact (Sterbenz), so no int->float conversion is needed.
__device__ __forceinline__ float uniform_f32(uint32_t x) {
    return mant_f32(x) - 0.99999994039535522f;
}

// Box-Muller pair scaled by the step noise: with bmc = -2 ln(2) sigma^2 and u1 from x0,
// R sigma = sqrt(bmc * log2(u1)).  The angle is formed from x1 in one multiply-add as
// 2 pi (1 + m 2^-23) - 3 pi = 2 pi (u2 - 2^-24) - pi, which lies in [-pi, pi) where the fast
// sincos is most accurate; the extra half turn is undone by returning the radius negated,
// rr = -R sigma, so the two noise increments are rr cos and rr sin -- the FP64 pair of the same
// words rotated by 2 pi 2^-24 (3.7e-7 rad), which leaves the Gaussian law unchanged.  They are
// returned as (rr, cos, sin) and the step multiplies them in an explicit fused multiply-add, so
// the rounding is the same in every kernel.  The radicand is taken in absolute value: the fast
// log2 can return a tiny positive value for u1 near 1.
__device__ __forceinline__ void bm_pair_f32(uint32_t x0, uint32_t x1, float bmc, float &rr,
                                            float &cs, float &sn) {
    const float u1 = uniform_f32(x0);
    rr = -sqrtf(fabsf(__fmul_rn(bmc, __log2f(u1))));
    __sincosf(fmaf(kTwoPiF, mant_f32(x1), -9.42477796076937972f), &sn, &cs);
}

// Double-precision uniform in (0, 1): u = (x + 1/2) 2^-32, exact.
__device__ __forceinline__ double uniform_f64(uint32_t x) {
    return __dmul_rn(__dadd_rn(static_cast<double>(x), 0.5), 2.3283064365386962890625e-10);
}

// Box-Muller in double precision, evaluated in the order R = sqrt(-2 log u1), theta = (2 pi) u2,
// z0 = R cos theta, z1 = R sin theta, each operation rounded separately.
__device__ __forceinline__ void bm_pair_f64(uint32_t x0, uint32_t x1, double &z0, double &z1) {
    const double u1 = uniform_f64(x0);
    const double u2 = uniform_f64(x1);
    const double r = __dsqrt_rn(__dmul_rn(-2.0, log(u1)));
    const double theta = __dmul_rn(6.283185307179586476925286766559, u2);
    z0 = __dmul_rn(r, cos(theta));
    z1 = __dmul_rn(r, sin(theta));
}

// Per-lane constants of the FP32 step, decoded from a request on the host (set-up of Alg. 1).
struct StepConstF32 {
    float dt;     // h
    float A;      // underdamped velocity coefficient: 1 - alpha dt (Euler), -alpha (Heun)
    float amp;    // amplitude of the sin term
    float bmc;    // -2 ln 2 sigma^2 (Box-Muller radius in log2 form)
    float nudt;   // bias increment per step (Alg. 3: delta-gamma)
};

enum : int { kUnder = 0, kOver = 1 };
enum : int { kEuler = 0, kHeun = 1 };
enum : int { kConstBias = 0, kRamp = 1 };

// Code path of a request: kind = model + 2 integrator + 4 ramp (eight paths).
__host__ __device__ constexpr int kind_of(int model, int integrator, int ramp) {
    return model + 2 * integrator + 4 * ramp;
}

// Bias arguments of the steps of a block.  Every FP32 step takes its bias already multiplied by
// dt, so bias and noise form addends that do not depend on the state (off the step's serial
// chain): the block's line is base = dt gs, slope = dt nu dt, and step s of the block
// (s = 0 .. kBlockSteps - 1) takes b0 = fmaf(slope, s, base) = dt gamma_{k-1} and
// b1 = fmaf(slope, s + kBiasEnd<H>, base): dt gamma_k for Euler, the midpoint
// dt (gamma_{k-1} + gamma_k) / 2 for Heun (s + 1/2 is exact).
template <int H>
constexpr float kBiasEnd = H == kHeun ? 0.5f : 1.0f;

__device__ __forceinline__ void bias_line(float gs, float nudt, float dt, float &base, float &slope) {
    base = __fmul_rn(dt, gs);
    slope = __fmul_rn(dt, nudt);
}

// Step s's bias arguments.  R = 1: the ramp of Alg. 3 (the line above).  R = 0: a constant bias
// (nu dt rounds to a zero slope), where both arguments are the base itself -- the value the
// line gives there (0 s + base = base), without the per-step multiply-add.  Every FP32 kernel
// selects R the same way (the ramp flag of the request's kind), so they agree bit for bit.
template <int H, int R>
__device__ __forceinline__ float bias_b0(float base, float slope, int s) {
    if constexpr (R) return fmaf(slope, static_cast<float>(s), base);
    else return base;
}
template <int H, int R>
__device__ __forceinline__ float bias_b1(float base, float slope, int s) {
    if constexpr (R) return fmaf(slope, static_cast<float>(s) + kBiasEnd<H>, base);
    else return base;
}

// One step with noise increment sigma z = rr * trig and dt-scaled bias b0, b1 (see bias_line);
// amp is the amplitude of the sin term, c = -amp dt, A the underdamped velocity coefficient.
// Euler-Maruyama (H = 0; Alg. 1 / Alg. 3, both updates read the state of the previous step;
// b1 = dt gamma_k):
//   underdamped: v' = (A v + (b1 + sigma z)) + c sin phi;  phi' = phi + v dt      [A = 1 - alpha dt]
//   overdamped : phi' = (phi + (b1 + sigma z)) + c sin phi
// Stochastic Heun (H = 1; predictor with the step's normal, corrector averaging the drift over
// both ends of the step; b0 = dt gamma_{k-1}, b1 = dt (gamma_{k-1} + gamma_k) / 2):
//   overdamped : p = (phi + (b0 + sigma z)) + c sin phi
//                phi' = (phi + (b1 + sigma z)) + (c / 2) (sin phi + sin p)
//   underdamped: q = ((v + (b0 + sigma z)) + (A dt) v) + c sin phi;  p = phi + v dt
//                v' = ((v + (b1 + sigma z)) + (A dt / 2)(v + q)) + (c / 2)(sin phi + sin p)
//                phi' = phi + (dt / 2)(v + q)                                       [A = -alpha]
//   i.e. a0 = A v - amp sin phi + gamma_{k-1}, q = v + a0 dt + sigma z,
//   a1 = A q - amp sin p + gamma_k, v' = v + (a0 + a1) dt / 2 + sigma z.
// r is the phase wrapped to [-pi, pi); the caller restores the range and counts windings.
// Every rounding is explicit (fmaf / __fmul_rn / __fadd_rn), so all kernels that take this step
// agree bit for bit.
template <int M, int H>
__device__ __forceinline__ void step_f32(float &r, float &v, float rr, float trig, float b0,
                                         float b1, float dt, float A, float amp) {
    const float c = __fmul_rn(-amp, dt);
    if constexpr (H == kEuler) {
        const float s = __sinf(r);
        const float q = fmaf(rr, trig, b1);    // dt gamma_k + sigma z: independent of the state
        if constexpr (M == kUnder) {
            const float vn = fmaf(c, s, fmaf(A, v, q));
            r = fmaf(dt, v, r);
            v = vn;
        } else {
            r = fmaf(c, s, __fadd_rn(r, q));
        }
    } else {
        const float hc = __fmul_rn(0.5f, c);
        const float q0 = fmaf(rr, trig, b0);
        const float qm = fmaf(rr, trig, b1);
        const float s0 = __sinf(r);
        if constexpr (M == kUnder) {
            const float dA = __fmul_rn(dt, A);
            const float hdA = __fmul_rn(0.5f, dA);
            const float hdt = __fmul_rn(0.5f, dt);
            const float q = fmaf(c, s0, fmaf(dA, v, __fadd_rn(v, q0)));
            const float p = fmaf(dt, v, r);
            const float vq = __fadd_rn(v, q);
            const float s1 = __sinf(p);
            v = fmaf(hc, __fadd_rn(s0, s1), fmaf(hdA, vq, __fadd_rn(v, qm)));
            r = fmaf(hdt, vq, r);
        } else {
            const float p = fmaf(c, s0, __fadd_rn(r, q0));
            const float s1 = __sinf(p);
            r = fmaf(hc, __fadd_rn(s0, s1), __fadd_rn(r, qm));
        }
    }
}

}  // namespace fpt
