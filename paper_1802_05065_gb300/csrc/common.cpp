// common.cpp -- request decoding (the set-up of Alg. 1 and Alg. 3), exact-sum results and
// error strings.  Host code; built with floating-point contraction off so every double
// expression rounds as written.
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "internal.h"

namespace fpt {

namespace {
thread_local std::string t_error;
}

void set_error(const std::string &msg) { t_error = msg; }
const std::string &get_error() { return t_error; }

static bool finite(double x) { return std::isfinite(x); }

bool decode(const fpt_params *p, Decoded *d, std::string *err) {
    auto fail = [&](const char *m) {
        *err = m;
        return false;
    };
    if (!p) return fail("params is NULL");
    if (p->model != FPT_UNDERDAMPED && p->model != FPT_OVERDAMPED) return fail("unknown model");
    if (p->output != FPT_OUT_TIME && p->output != FPT_OUT_BIAS) return fail("unknown output");
    if (p->integrator != FPT_EULER_MARUYAMA && p->integrator != FPT_HEUN)
        return fail("unknown integrator");
    if (p->threshold_mode != FPT_TH_ABSOLUTE && p->threshold_mode != FPT_TH_FROM_START)
        return fail("unknown threshold_mode");
    if (!(p->dt > 0) || !finite(p->dt)) return fail("dt must be positive and finite");
    if (!(p->D >= 0) || !finite(p->D)) return fail("D must be >= 0");
    if (p->model == FPT_UNDERDAMPED && (!(p->alpha >= 0) || !finite(p->alpha)))
        return fail("alpha must be >= 0");
    if (!finite(p->gamma0) || !finite(p->nu) || !finite(p->sin_amp) || !finite(p->v0) ||
        !finite(p->threshold))
        return fail("non-finite parameter");
    if (p->max_steps < 1 || p->max_steps > kMaxSteps) return fail("max_steps must be in [1, 2^48]");
    if (p->hist_bins < 1 || p->hist_bins > kMaxBins) return fail("hist_bins must be in [1, 2^20]");
    if (!finite(p->hist_lo) || !finite(p->hist_hi) || !(p->hist_hi > p->hist_lo))
        return fail("need hist_lo < hist_hi");
    if (!(p->stop_rse >= 0) || !finite(p->stop_rse)) return fail("stop_rse must be >= 0");
    if (std::isnan(p->phi0) && !(std::fabs(p->gamma0) <= 1.0))
        return fail("phi0 = NaN needs |gamma0| <= 1 (phi0 = arcsin gamma0)");
    if (!std::isnan(p->phi0) && !finite(p->phi0)) return fail("phi0 must be finite or NaN");

    d->model = p->model;
    d->integrator = p->integrator;
    d->output = p->output;
    d->alpha = p->model == FPT_UNDERDAMPED ? p->alpha : 0.0;
    d->D = p->D;
    d->gamma0 = p->gamma0;
    d->nudt = p->nu * p->dt;
    d->amp = p->sin_amp;
    d->dt = p->dt;
    d->sigma = p->model == FPT_UNDERDAMPED ? std::sqrt(2.0 * p->alpha * p->D * p->dt)
                                           : std::sqrt(2.0 * p->D * p->dt);
    d->phi0 = std::isnan(p->phi0) ? std::asin(p->gamma0) : p->phi0;
    d->v0 = p->model == FPT_UNDERDAMPED ? p->v0 : 0.0;
    d->th = p->threshold_mode == FPT_TH_FROM_START ? d->phi0 + p->threshold : p->threshold;
    if (!(d->th > d->phi0)) return fail("threshold must lie above the start phase");
    d->max_steps = p->max_steps;
    d->out_a = p->output == FPT_OUT_TIME ? 0.0 : p->gamma0;
    d->out_b = p->output == FPT_OUT_TIME ? p->dt : d->nudt;
    d->hist_bins = p->hist_bins;
    d->hist_lo = p->hist_lo;
    d->hist_hi = p->hist_hi;
    d->hist_inv_w = static_cast<double>(p->hist_bins) / (p->hist_hi - p->hist_lo);

    // single precision
    d->dt_f = static_cast<float>(d->dt);
    d->A_f = d->integrator == FPT_HEUN ? static_cast<float>(-d->alpha)
                                       : static_cast<float>(1.0 - d->alpha * d->dt);
    d->amp_f = static_cast<float>(d->amp);
    d->bmc_f = static_cast<float>(-2.0 * M_LN2 * d->sigma * d->sigma);
    d->nudt_f = static_cast<float>(d->nudt);
    // code path: model, integrator, and whether the single-precision bias ramps at all
    d->kind = p->model + 2 * p->integrator + 4 * (d->nudt_f != 0.0f ? 1 : 0);
    d->v0_f = static_cast<float>(d->v0);
    const double two_pi = 2.0 * M_PI;
    double w0 = std::floor((d->phi0 + M_PI) / two_pi);
    double r0 = d->phi0 - two_pi * w0;
    float r0f = static_cast<float>(r0);
    if (r0f >= static_cast<float>(M_PI)) {
        r0f -= static_cast<float>(two_pi);
        w0 += 1.0;
    }
    if (r0f < -static_cast<float>(M_PI)) r0f = -static_cast<float>(M_PI);
    if (std::fabs(w0) > 1e6) return fail("start phase too far from 0");
    d->r0_f = r0f;
    d->w0 = static_cast<int32_t>(w0);
    d->eb0_f = static_cast<float>(d->th - two_pi * w0);
    return true;
}

// 128-bit helpers (GCC/Clang on x86-64 and aarch64).
using u128 = unsigned __int128;
using i128 = __int128;

static double u128_to_double(u128 x) {
    return static_cast<double>(static_cast<uint64_t>(x >> 64)) * 18446744073709551616.0 +
           static_cast<double>(static_cast<uint64_t>(x));
}

// Mean and unbiased variance of x = a + b k from exact integer sums of k and k^2:
// centred at the integer mean c, M2 = sum (k - c)^2 = s2 - 2 c s1 + n c^2 exactly, then
// var_k = (M2 - (s1 - n c)^2 / n) / (n - 1).
void sums_to_result(const Decoded &d, const fpt_sums &s, fpt_result *out) {
    const uint64_t n = s.n_escaped;
    out->n_escaped = n;
    out->n_censored = s.n_done - n;
    out->mean = out->var = out->sem = NAN;
    if (n == 0) return;
    const u128 s1 = (static_cast<u128>(s.s1_hi) << 64) | s.s1_lo;
    const u128 s2 = (static_cast<u128>(s.s2_hi) << 64) | s.s2_lo;
    const u128 c = s1 / n;
    const double mean_k = u128_to_double(c) + u128_to_double(s1 - c * n) / static_cast<double>(n);
    out->mean = d.output == FPT_OUT_TIME ? d.out_b * mean_k : d.out_a + d.out_b * mean_k;
    if (n < 2) return;
    // M2 = s2 - 2 c s1 + n c^2.  With s1 < 2^76 and c < 2^48 every term is below 2^126
    // (s2 <= max k * s1 < 2^124); larger sums fall back to double arithmetic.
    double var_k;
    const bool small = (s1 >> 76) == 0 && (c >> 48) == 0;
    if (small) {
        const i128 m2 = static_cast<i128>(s2) - static_cast<i128>(2 * c * s1) +
                        static_cast<i128>(c * c * n);
        const i128 dev = static_cast<i128>(s1) - static_cast<i128>(c * n);   // 0 <= dev < n
        const double devd = static_cast<double>(static_cast<int64_t>(dev));
        const double m2d = m2 >= 0 ? u128_to_double(static_cast<u128>(m2)) : 0.0;
        var_k = (m2d - devd * devd / static_cast<double>(n)) / static_cast<double>(n - 1);
    } else {
        const double s1d = u128_to_double(s1), s2d = u128_to_double(s2);
        var_k = (s2d - s1d * (s1d / static_cast<double>(n))) / static_cast<double>(n - 1);
    }
    if (var_k < 0) var_k = 0;
    out->var = d.out_b * d.out_b * var_k;
    out->sem = std::sqrt(out->var / static_cast<double>(n));
}

}  // namespace fpt

using namespace fpt;

extern "C" fpt_status fpt_sums_finish(const fpt_params *params, const fpt_sums *sums,
                                      fpt_result *out) {
    Decoded d;
    std::string err;
    if (!sums || !out) {
        set_error("NULL argument");
        return FPT_EINVAL;
    }
    if (!decode(params, &d, &err)) {
        set_error(err);
        return FPT_EINVAL;
    }
    std::memset(out, 0, sizeof(*out));
    out->state = FPT_OK;
    out->n_used = sums->n_done;
    sums_to_result(d, *sums, out);
    const u128 s1 = (static_cast<u128>(sums->s1_hi) << 64) | sums->s1_lo;
    const u128 tot = s1 + static_cast<u128>(sums->n_done - sums->n_escaped) * d.max_steps;
    out->steps_total = tot >> 64 ? UINT64_MAX : static_cast<uint64_t>(tot);
    return FPT_OK;
}

extern "C" const char *fpt_status_string(fpt_status s) {
    switch (s) {
        case FPT_OK: return "ok";
        case FPT_PENDING: return "pending";
        case FPT_EINVAL: return "invalid argument";
        case FPT_ENOMEM: return "out of device memory or budget";
        case FPT_EBUSY: return "busy";
        case FPT_ENOTFOUND: return "request not found";
        case FPT_ETIMEDOUT: return "timed out";
        case FPT_ECUDA: return "CUDA error";
        case FPT_EFULL: return "queue full";
    }
    return "unknown status";
}

extern "C" const char *fpt_version(void) { return "fpt-gb300 0.1 (sm_103a)"; }

// ---- paper units (Sec. II.A, Eq. JJn) <-> engine units ----------------------------------------
// The paper's time unit is hbar / E_C; rescaling time by sqrt(V0) (V0 = E_J / E_C) gives the
// plasma-frequency units of the engine.  Arithmetic in IEEE double, contraction off.

static bool positive_finite(double x) { return std::isfinite(x) && x > 0; }

extern "C" fpt_status fpt_from_paper_units(double V0, double beta, double theta, double h,
                                           double delta_gamma, double *alpha, double *D,
                                           double *dt, double *nu) {
    if (!alpha || !D || !dt || !nu) {
        set_error("NULL output");
        return FPT_EINVAL;
    }
    if (!positive_finite(V0) || !positive_finite(h) || !std::isfinite(beta) || !std::isfinite(theta) ||
        !std::isfinite(delta_gamma)) {
        set_error("V0 and h must be positive; beta, theta, delta_gamma finite");
        return FPT_EINVAL;
    }
    const double s = std::sqrt(V0);
    *dt = s * h;
    *alpha = beta / s;
    *D = theta / V0;
    *nu = delta_gamma / *dt;
    return FPT_OK;
}

extern "C" fpt_status fpt_to_paper_units(double alpha, double D, double dt, double nu, double V0,
                                         double *beta, double *theta, double *h,
                                         double *delta_gamma) {
    if (!beta || !theta || !h || !delta_gamma) {
        set_error("NULL output");
        return FPT_EINVAL;
    }
    if (!positive_finite(V0) || !positive_finite(dt) || !std::isfinite(alpha) || !std::isfinite(D) ||
        !std::isfinite(nu)) {
        set_error("V0 and dt must be positive; alpha, D, nu finite");
        return FPT_EINVAL;
    }
    const double s = std::sqrt(V0);
    *h = dt / s;
    *beta = alpha * s;
    *theta = D * V0;
    *delta_gamma = nu * dt;
    return FPT_OK;
}

extern "C" fpt_status fpt_junction_paper_units(double R, double C, double Ic, double T, double *V0,
                                               double *beta, double *theta, double *time_unit_s) {
    if (!V0 || !beta || !theta || !time_unit_s) {
        set_error("NULL output");
        return FPT_EINVAL;
    }
    if (!positive_finite(R) || !positive_finite(C) || !positive_finite(Ic) || !(T >= 0) ||
        !std::isfinite(T)) {
        set_error("R, C, Ic must be positive and T >= 0");
        return FPT_EINVAL;
    }
    const double hbar = 1.054571817e-34, e_charge = 1.602176634e-19, k_b = 1.380649e-23;   // SI
    const double two_e = 2.0 * e_charge;
    const double e_j = hbar * Ic / two_e;        // Josephson energy
    const double e_c = two_e * two_e / C;        // charging energy of a Cooper pair
    *V0 = e_j / e_c;
    *beta = hbar / (R * two_e * two_e);
    *theta = k_b * T / e_c;
    *time_unit_s = hbar / e_c;
    return FPT_OK;
}

extern "C" fpt_status fpt_sweep_delta_gamma(double sweep_hz, double h, double time_unit_s, double span,
                                            double *delta_gamma) {
    if (!delta_gamma) {
        set_error("NULL output");
        return FPT_EINVAL;
    }
    if (!positive_finite(sweep_hz) || !positive_finite(h) || !positive_finite(time_unit_s) ||
        !std::isfinite(span)) {
        set_error("sweep_hz, h and time_unit_s must be positive, span finite");
        return FPT_EINVAL;
    }
    const double ramp_time_s = 0.5 / sweep_hz;   // half a period of a triangular sweep
    *delta_gamma = span / (ramp_time_s / (h * time_unit_s));
    return FPT_OK;
}
