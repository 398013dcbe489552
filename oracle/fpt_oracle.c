/*
 * fpt_oracle.c -- plain FP64 CPU oracle for the first-passage-time (FPT) method of
 * "Stochastic first passage time accelerated with CUDA" (Pierro, Troiano, Mejuto, Filatrella).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker, not the product: only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg may load it.  It shares no code, header,
 * table or constant generator with the CUDA engine; it is written from the paper and from the
 * published definition of Philox4x32-10, step by step, with no blocking or reordering.
 *
 * Build: cc -O2 -ffp-contract=off [-fopenmp] -shared -fPIC.  Floating-point contraction must be
 * off so that every product and sum below is rounded exactly as written.
 *
 * What it computes (all in IEEE double, unwrapped phase):
 *   - Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of two 32x32->64 multiplies
 *     with multipliers 0xD2511F53 / 0xCD9E8D57 and a Weyl key schedule 0x9E3779B9 / 0xBB67AE85.
 *   - Box-Muller normals (Sec. III.B, the nrand function of Alg. 1 and Alg. 3): basic form,
 *     both outputs used, cosine first.
 *   - The Euler-Maruyama step of Alg. 1 (constant bias) and Alg. 3 (ramped bias), underdamped
 *     form of Eq. (JJn) in plasma-frequency units, phi'' + alpha phi' + sin phi = gamma + noise,
 *     and its overdamped counterpart phi' = gamma - sin phi + noise.
 *   - The stochastic Heun predictor-corrector on the same model (one normal per step, drift
 *     averaged over both ends of the step; Kloeden-Platen's weak order-2 scheme for additive
 *     noise).  The paper integrates with the Euler scheme only (Sec. III); Heun is an option
 *     of this implementation, pinned on its own closed forms.
 *   - The first step index k at which phi_k >= threshold (escape), or censoring at max_steps.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ----------------------------------------------------------------------------------------------
 * Philox4x32-10.  One round maps counter (c0,c1,c2,c3) under round key (k0,k1) to
 *   (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0)),
 * and the key is advanced by the Weyl constants between rounds.
 * -------------------------------------------------------------------------------------------- */
#define ORACLE_PHILOX_M0 0xD2511F53u
#define ORACLE_PHILOX_M1 0xCD9E8D57u
#define ORACLE_PHILOX_W0 0x9E3779B9u
#define ORACLE_PHILOX_W1 0xBB67AE85u

void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)ORACLE_PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)ORACLE_PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += ORACLE_PHILOX_W0;
        k1 += ORACLE_PHILOX_W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Random-number keying of one trajectory (reading of the paper's per-thread seeding, Sec. III.B):
 * key = (seed low word, seed high word); counter = (block low, block high, trajectory low,
 * trajectory high), where block b holds the normals of steps 4b+1 .. 4b+4. */
void oracle_philox_block(uint64_t seed, uint64_t traj, uint64_t block, uint32_t out[4])
{
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t ctr[4] = { (uint32_t)block, (uint32_t)(block >> 32), (uint32_t)traj,
                        (uint32_t)(traj >> 32) };
    oracle_philox4x32_10(ctr, key, out);
}

/* Uniform deviate in the open interval (0,1): u = (x + 1/2) / 2^32, exact in double.
 * The paper maps the 32-bit integer linearly to [0,1] (Sec. III.B); the half offset keeps
 * u away from 0 so that log(u) is finite. */
double oracle_uniform(uint32_t x)
{
    return ((double)x + 0.5) * (1.0 / 4294967296.0);
}

/* Box-Muller transform (nrand, Sec. III.B): R = sqrt(-2 ln u1), theta = 2 pi u2,
 * z0 = R cos theta, z1 = R sin theta. */
void oracle_box_muller(uint32_t x0, uint32_t x1, double *z0, double *z1)
{
    double u1 = oracle_uniform(x0);
    double u2 = oracle_uniform(x1);
    double r = sqrt(-2.0 * log(u1));
    double theta = (2.0 * M_PI) * u2;
    *z0 = r * cos(theta);
    *z1 = r * sin(theta);
}

/* The n-th standard normal (n = 0, 1, 2, ...) of trajectory `traj`: block n/4, slot n%4,
 * slots (0,1) from words (x0,x1) and slots (2,3) from words (x2,x3). */
double oracle_normal(uint64_t seed, uint64_t traj, uint64_t n)
{
    uint32_t x[4];
    double z[4];
    oracle_philox_block(seed, traj, n / 4, x);
    oracle_box_muller(x[0], x[1], &z[0], &z[1]);
    oracle_box_muller(x[2], x[3], &z[2], &z[3]);
    return z[n % 4];
}

/* ----------------------------------------------------------------------------------------------
 * Model parameters.  Own definition (not shared with the engine's ABI header).
 * -------------------------------------------------------------------------------------------- */
typedef struct {
    int32_t model;          /* 0 = underdamped (Eq. JJn), 1 = overdamped */
    int32_t threshold_mode; /* 0 = absolute phi*, 1 = phi0 + threshold */
    int32_t integrator;     /* 0 = Euler-Maruyama (Alg. 1), 1 = stochastic Heun */
    int32_t reserved;
    double alpha;           /* damping (the paper's beta in plasma-frequency units) */
    double D;               /* noise intensity k_B T / E_J */
    double gamma0;          /* bias at k = 0 */
    double nu;              /* bias ramp per unit time (Alg. 3: delta-gamma per step = nu*dt) */
    double sin_amp;         /* amplitude of the sin phi term: 1 for the junction, 0 = free drift */
    double dt;              /* Euler step h */
    double phi0;            /* start phase; NaN means arcsin(gamma0) (Alg. 1 / Alg. 3) */
    double v0;              /* start velocity (underdamped only) */
    double threshold;       /* phi* (absolute) or offset from phi0 */
    uint64_t max_steps;     /* klim of Alg. 1; reaching it without escape = censored */
} oracle_params;

/* Noise amplitude per step.  Underdamped: the fluctuation-dissipation-consistent reading of
 * Alg. 1's sigma = sqrt(2 D h) in units where damping alpha multiplies the velocity:
 * sigma = sqrt(2 alpha D dt).  Overdamped: sigma = sqrt(2 D dt). */
double oracle_sigma(const oracle_params *p)
{
    if (p->model == 0) return sqrt(2.0 * p->alpha * p->D * p->dt);
    return sqrt(2.0 * p->D * p->dt);
}

double oracle_start_phase(const oracle_params *p)
{
    if (isnan(p->phi0)) return asin(p->gamma0);
    return p->phi0;
}

double oracle_threshold(const oracle_params *p)
{
    if (p->threshold_mode == 1) return oracle_start_phase(p) + p->threshold;
    return p->threshold;
}

/* One trajectory, Alg. 1 (nu = 0) or Alg. 3 (nu != 0), in FP64 with an unwrapped phase.
 * Step k (k = 1, 2, ...), Euler-Maruyama:
 *   gamma_k = gamma0 + (nu*dt)*k                   (Alg. 3 sets gamma_k before the update)
 *   underdamped:  phi_k = phi_{k-1} + v_{k-1}*dt
 *                 v_k   = v_{k-1} + (-alpha*v_{k-1} - A*sin(phi_{k-1}) + gamma_k)*dt + sigma*z_k
 *   overdamped:   phi_k = phi_{k-1} + (gamma_k - A*sin(phi_{k-1}))*dt + sigma*z_k
 * Stochastic Heun (predictor-corrector with the same z_k; drift at both ends of the step, the
 * bias taken at t_{k-1} and t_k):
 *   overdamped:   f0 = gamma_{k-1} - A sin(phi);  p = phi + f0*dt + sigma*z
 *                 f1 = gamma_k - A sin(p);         phi_k = phi + ((f0 + f1)*0.5)*dt + sigma*z
 *   underdamped:  a0 = -alpha*v - A sin(phi) + gamma_{k-1};  p = phi + v*dt;  q = v + a0*dt + sigma*z
 *                 a1 = -alpha*q - A sin(p) + gamma_k
 *                 phi_k = phi + ((v + q)*0.5)*dt;  v_k = v + ((a0 + a1)*0.5)*dt + sigma*z
 * Escape when phi_k >= threshold: return k.  If k reaches max_steps first: censored.
 * Returns 1 for escape (k_out = escape step) and 0 for censored (k_out = max_steps).
 * If trace_phi / trace_v are non-NULL they receive phi_k, v_k for k = 1..min(k, trace_len). */
int oracle_trajectory_trace(const oracle_params *p, uint64_t seed, uint64_t traj,
                            uint64_t *k_out, double *phi_end, double *v_end,
                            double *trace_phi, double *trace_v, uint64_t trace_len)
{
    const double sigma = oracle_sigma(p);
    const double th = oracle_threshold(p);
    const double nudt = p->nu * p->dt;
    double phi = oracle_start_phase(p);
    double v = p->v0;
    double z[4] = {0.0, 0.0, 0.0, 0.0};
    uint64_t k = 0;
    int escaped = 0;
    while (k < p->max_steps) {
        uint64_t n = k;  /* index of the normal used by step k+1 */
        if (n % 4 == 0) {
            uint32_t x[4];
            oracle_philox_block(seed, traj, n / 4, x);
            oracle_box_muller(x[0], x[1], &z[0], &z[1]);
            oracle_box_muller(x[2], x[3], &z[2], &z[3]);
        }
        double zk = z[n % 4];
        k = k + 1;
        double g = p->gamma0 + nudt * (double)k;
        double s = sin(phi);
        double phi_new, v_new;
        if (p->integrator == 1) {
            double g0 = p->gamma0 + nudt * (double)(k - 1);
            if (p->model == 0) {
                double a0 = -p->alpha * v - p->sin_amp * s + g0;
                double pp = phi + v * p->dt;
                double q = v + a0 * p->dt + sigma * zk;
                double a1 = -p->alpha * q - p->sin_amp * sin(pp) + g;
                phi_new = phi + ((v + q) * 0.5) * p->dt;
                v_new = v + ((a0 + a1) * 0.5) * p->dt + sigma * zk;
            } else {
                double f0 = g0 - p->sin_amp * s;
                double pp = phi + f0 * p->dt + sigma * zk;
                double f1 = g - p->sin_amp * sin(pp);
                phi_new = phi + ((f0 + f1) * 0.5) * p->dt + sigma * zk;
                v_new = 0.0;
            }
        } else if (p->model == 0) {
            phi_new = phi + v * p->dt;
            v_new = v + (-p->alpha * v - p->sin_amp * s + g) * p->dt + sigma * zk;
        } else {
            phi_new = phi + (g - p->sin_amp * s) * p->dt + sigma * zk;
            v_new = 0.0;
        }
        phi = phi_new;
        v = v_new;
        if (trace_phi && k <= trace_len) trace_phi[k - 1] = phi;
        if (trace_v && k <= trace_len) trace_v[k - 1] = v;
        if (phi >= th) { escaped = 1; break; }
    }
    *k_out = k;
    if (phi_end) *phi_end = phi;
    if (v_end) *v_end = v;
    return escaped;
}

int oracle_trajectory(const oracle_params *p, uint64_t seed, uint64_t traj, uint64_t *k_out)
{
    return oracle_trajectory_trace(p, seed, traj, k_out, NULL, NULL, NULL, NULL, 0);
}

/* Many independent realisations (the paper's T_e array, Sec. III.A): trajectory ids
 * id0 .. id0+n-1, one after another; OpenMP only distributes whole trajectories.
 * steps[i] = escape step, or -1 if censored (Alg. 1's -1 sentinel). */
void oracle_run(const oracle_params *p, uint64_t seed, uint64_t id0, uint64_t n,
                int64_t *steps, int nthreads)
{
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#else
    (void)nthreads;
#endif
    for (int64_t i = 0; i < (int64_t)n; ++i) {
        uint64_t k = 0;
        int esc = oracle_trajectory(p, seed, id0 + (uint64_t)i, &k);
        steps[i] = esc ? (int64_t)k : -1;
    }
}

/* Run selected trajectory ids (for sampled comparison of a large launch). */
void oracle_run_ids(const oracle_params *p, uint64_t seed, const uint64_t *ids, uint64_t n,
                    int64_t *steps, int nthreads)
{
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#else
    (void)nthreads;
#endif
    for (int64_t i = 0; i < (int64_t)n; ++i) {
        uint64_t k = 0;
        int esc = oracle_trajectory(p, seed, ids[i], &k);
        steps[i] = esc ? (int64_t)k : -1;
    }
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
