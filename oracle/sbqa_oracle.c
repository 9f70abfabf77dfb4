/*
 * sbqa_oracle.c -- plain FP64 CPU oracle of the SBQA hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * restatement of Simulated Bifurcation Quantum Annealing (Pawlowski et al.,
 * "Simulated Bifurcation Quantum Annealing", arXiv 2604.01050) that the CUDA
 * library is checked against.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load it.  It shares no code, header or
 * table with the CUDA library; the two agree only through the paper.
 *
 * Notation (the paper writes R for the Trotter replicas of one run; here the
 * replicas of one run are P and the independent runs are R):
 *   N spins i, P Trotter replicas k (periodic ring), R independent runs r,
 *   S steps n, tau_n = n / S (= t / T).
 * State arrays are run-major: x[(r * P + k) * N + i].
 *
 * What each function follows:
 *   orc_splitmix64      SplitMix64 (Steele, Lea & Flood 2014): output number
 *                       ctr of the generator seeded with seed.
 *   orc_init_state      random initial state ("initialized in a random
 *                       state", Sec. II A), read through SplitMix64.
 *   orc_schedule        a(t) = t/T (Sec. II A, after Eq. 2); Gamma_x(t) and
 *                       J_perp(t) (Sec. II A, Eq. 5; Supplement Eq. S12);
 *                       Delta(t) = 0.7 t/T (Sec. II A, after Eq. 8).
 *   orc_f               thresholded f of Eq. 8 (dSB-type) or f(x)=x (bSB,
 *                       Sec. II A after Eq. 3).
 *   orc_force/orc_run   SBQA equations of motion, Eqs. 6-7, integrated by
 *                       symplectic Euler (momentum first, then position),
 *                       followed by the wall rule stated after Eq. 3.
 *   orc_energy          Ising energy E(s) = -sum_{i<j} J_ij s_i s_j
 *                       - sum_i h_i s_i, the sign convention of the SBQA
 *                       Hamiltonian Eq. 4 and of H_Q in Supplement Eq. S1.
 *   orc_readout         s = sign(q) (Sec. II A), best over replicas and runs
 *                       ("return the best solution", Sec. II B).
 *   orc_brute_force     exhaustive ground state for small N.
 *   orc_round_bf16      round-to-nearest-even of a double to bfloat16 (the
 *                       documented quantisation of J for the BF16 product).
 *
 * Readings where the paper is silent:
 *   - integrator: symplectic Euler, y from x(t_n) first, x from the new y,
 *     then the wall; step n uses tau_n = n/S;
 *   - f at the threshold: |x| <= Delta gives 0 (inclusive), compared in
 *     FP64 like every other step of this file;
 *   - readout sign: x >= 0 gives +1;
 *   - wall: strict |x| > 1 after the position update, then x <- sign(x),
 *     y <- 0;
 *   - replicas k-1, k+1 are taken modulo P (periodic imaginary time,
 *     Supplement Eq. S3 boundary condition).
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -shared -fPIC (no FMA
 * contraction, so x86 and Arm hosts give the same bits).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* SplitMix64: state advances by the golden gamma, output is the       */
/* variant-13 finaliser of the state (Steele, Lea & Flood, OOPSLA 2014) */
/* ------------------------------------------------------------------ */
uint64_t orc_splitmix64(uint64_t seed, uint64_t ctr)
{
    uint64_t z = seed + (ctr + 1u) * 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

/* Map a 64-bit output to an FP32 value in [-amp, amp):
 * m = top 24 bits - 2^23, u = m * 2^-23 (exact in FP32), v = fl32(u * amp). */
float orc_uniform_f32(uint64_t z, float amp)
{
    int32_t m = (int32_t)(z >> 40) - 8388608;
    float u = (float)m * 0x1p-23f;
    return u * amp;
}

/* Initial state of Sec. II A.  Counter of element (r, k, i), component
 * w (0 = position x, 1 = momentum y):
 *   ctr = (((r * P + k) * N + i) * 2 + w). */
void orc_init_state(uint64_t seed, int N, int P, int R, double amp,
                    double *x, double *y)
{
    float amp_f = (float)amp;
    for (int r = 0; r < R; ++r)
        for (int k = 0; k < P; ++k)
            for (int i = 0; i < N; ++i) {
                uint64_t e = ((uint64_t)r * (uint64_t)P + (uint64_t)k) * (uint64_t)N + (uint64_t)i;
                x[e] = (double)orc_uniform_f32(orc_splitmix64(seed, 2u * e + 0u), amp_f);
                y[e] = (double)orc_uniform_f32(orc_splitmix64(seed, 2u * e + 1u), amp_f);
            }
}

/* ------------------------------------------------------------------ */
/* bfloat16 rounding: 8 significant bits, round to nearest, ties even  */
/* ------------------------------------------------------------------ */
double orc_round_bf16(double v)
{
    if (v == 0.0 || !isfinite(v)) return v;
    int e;
    double m = frexp(v, &e);          /* v = m * 2^e, 0.5 <= |m| < 1 */
    double q = nearbyint(ldexp(m, 8)); /* 8 significant bits, RNE */
    return ldexp(q, e - 8);
}

/* ------------------------------------------------------------------ */
/* Schedule (Sec. II A)                                                */
/* ------------------------------------------------------------------ */
/* J_perp = -(1/(2 beta)) ln tanh(beta Gamma / P)   (Eq. 5, Eq. S12) */
double orc_jperp(double beta, double gamma, int P)
{
    return -log(tanh(beta * gamma / (double)P)) / (2.0 * beta);
}

/* Gamma_x(t) = Gamma_x(0) [ (1 - t/T)^alpha + 1e-5 ]   (Eq. 5) */
double orc_gamma(double gamma0, double alpha, double tau)
{
    return gamma0 * (pow(1.0 - tau, alpha) + 1e-5);
}

/* Tables for steps n = 0..S-1 (the threshold table has S+1 entries, the
 * extra one being tau = 1, used nowhere in the dynamics):
 *   a[n] = tau_n, delta[n] = delta_slope * tau_n,
 *   jperp[r * S + n] = J_perp(beta_r, Gamma_x(tau_n; alpha_r))  (0 if disabled). */
void orc_schedule(int S, int P, int R, double gamma0, double delta_slope,
                  const double *beta, const double *alpha, int jperp_enable,
                  double *a, double *delta, double *jperp)
{
    for (int n = 0; n <= S; ++n) {
        double tau = (double)n / (double)S;
        if (n < S) a[n] = tau;
        delta[n] = delta_slope * tau;
    }
    for (int r = 0; r < R; ++r)
        for (int n = 0; n < S; ++n) {
            double tau = (double)n / (double)S;
            jperp[(size_t)r * S + n] =
                jperp_enable ? orc_jperp(beta[r], orc_gamma(gamma0, alpha[r], tau), P) : 0.0;
        }
}

/* ------------------------------------------------------------------ */
/* Problem: J as CSR (a dense J is passed with every off-diagonal entry) */
/* ------------------------------------------------------------------ */
typedef struct {
    int n;
    const int64_t *row_ptr; /* n + 1 */
    const int32_t *col;     /* nnz */
    const double *val;      /* nnz */
    const double *h;        /* n, may be NULL */
} orc_problem;

/* c0 default: 0.5 * sqrt(N / sum_ij J_ij^2) (Goto et al. 2021 choice,
 * written with the rms row norm so that it also covers sparse J). */
double orc_c0_auto(const orc_problem *pb)
{
    double s2 = 0.0;
    int64_t nnz = pb->row_ptr[pb->n];
    for (int64_t e = 0; e < nnz; ++e) s2 += pb->val[e] * pb->val[e];
    if (s2 <= 0.0) return 0.5;
    return 0.5 * sqrt((double)pb->n / s2);
}

/* f of Eq. 8 (variant 0) or the bSB choice f(x) = x (variant 1). */
double orc_f(double x, double delta, int variant)
{
    if (variant == 1) return x;
    if (fabs(x) <= delta) return 0.0;
    return x > 0.0 ? 1.0 : -1.0;
}

typedef struct {
    double a0, c0, dt;
    int variant; /* 0: thresholded sign (Eq. 8), 1: f(x) = x */
} orc_params;

/* Force on every (k, i) of one run at step n (right-hand side of Eq. 7):
 *   F = -((a0 - a_n)/P) x_{i,k} + (c0/P) (sum_j J_ij f(x_{j,k}) + h_i)
 *       + J_perp (x_{i,k-1} + x_{i,k+1}).
 * x points at the run's P*N positions; out receives P*N forces. */
void orc_force(const orc_problem *pb, const orc_params *pp, int P,
               double a_n, double delta_n, double jperp, const double *x,
               double *out)
{
    int N = pb->n;
    double *fx = (double *)malloc(sizeof(double) * (size_t)P * (size_t)N);
    for (int k = 0; k < P; ++k)
        for (int j = 0; j < N; ++j)
            fx[(size_t)k * N + j] = orc_f(x[(size_t)k * N + j], delta_n, pp->variant);
    for (int k = 0; k < P; ++k) {
        int km = (k + P - 1) % P, kp = (k + 1) % P;
        for (int i = 0; i < N; ++i) {
            double g = 0.0;
            for (int64_t e = pb->row_ptr[i]; e < pb->row_ptr[i + 1]; ++e)
                g += pb->val[e] * fx[(size_t)k * N + pb->col[e]];
            double hi = pb->h ? pb->h[i] : 0.0;
            double xi = x[(size_t)k * N + i];
            out[(size_t)k * N + i] = -((pp->a0 - a_n) / (double)P) * xi
                                     + (pp->c0 / (double)P) * (g + hi)
                                     + jperp * (x[(size_t)km * N + i] + x[(size_t)kp * N + i]);
        }
    }
    free(fx);
}

/* One symplectic-Euler step of one run: y += dt F(x); x += dt (a0/P) y;
 * wall: if |x| > 1 then x = sign(x), y = 0  (rule stated after Eq. 3). */
void orc_step_run(const orc_problem *pb, const orc_params *pp, int P,
                  double a_n, double delta_n, double jperp, double *x, double *y)
{
    size_t M = (size_t)P * (size_t)pb->n;
    double *F = (double *)malloc(sizeof(double) * M);
    orc_force(pb, pp, P, a_n, delta_n, jperp, x, F);
    for (size_t e = 0; e < M; ++e) {
        y[e] = y[e] + pp->dt * F[e];
        x[e] = x[e] + pp->dt * (pp->a0 / (double)P) * y[e];
        if (fabs(x[e]) > 1.0) {
            x[e] = x[e] > 0.0 ? 1.0 : -1.0;
            y[e] = 0.0;
        }
    }
    free(F);
}

/* ------------------------------------------------------------------ */
/* Energies and readout                                                */
/* ------------------------------------------------------------------ */
/* E(s) = -sum_{i<j} J_ij s_i s_j - sum_i h_i s_i.  With symmetric J the
 * pair sum is half of the full double sum, which is what is added here. */
double orc_energy(const orc_problem *pb, const int8_t *s)
{
    double pair = 0.0, field = 0.0;
    for (int i = 0; i < pb->n; ++i) {
        for (int64_t e = pb->row_ptr[i]; e < pb->row_ptr[i + 1]; ++e) {
            int j = pb->col[e];
            if (j > i) pair += pb->val[e] * (double)s[i] * (double)s[j];
        }
        if (pb->h) field += pb->h[i] * (double)s[i];
    }
    return -pair - field;
}

/* Exact integer energy for integer-valued J and h (caller guarantees it). */
int64_t orc_energy_int(const orc_problem *pb, const int8_t *s)
{
    int64_t pair = 0, field = 0;
    for (int i = 0; i < pb->n; ++i) {
        for (int64_t e = pb->row_ptr[i]; e < pb->row_ptr[i + 1]; ++e) {
            int j = pb->col[e];
            if (j > i) pair += (int64_t)llround(pb->val[e]) * s[i] * s[j];
        }
        if (pb->h) field += (int64_t)llround(pb->h[i]) * s[i];
    }
    return -pair - field;
}

/* s = sign(q) with q >= 0 giving +1. */
void orc_sign(const double *x, int8_t *s, size_t m)
{
    for (size_t e = 0; e < m; ++e) s[e] = x[e] >= 0.0 ? 1 : -1;
}

/* Exhaustive minimum of E over all 2^N spin vectors (N <= 30).
 * Returns the minimum; writes one minimiser (the first in counting order,
 * bit i of the counter set meaning s_i = -1). */
double orc_brute_force(const orc_problem *pb, int8_t *best_s)
{
    int N = pb->n;
    int8_t *s = (int8_t *)malloc((size_t)N);
    double best = INFINITY;
    uint64_t count = 1ull << N;
    for (uint64_t b = 0; b < count; ++b) {
        for (int i = 0; i < N; ++i) s[i] = ((b >> i) & 1u) ? -1 : 1;
        double e = orc_energy(pb, s);
        if (e < best) {
            best = e;
            if (best_s) memcpy(best_s, s, (size_t)N);
        }
    }
    free(s);
    return best;
}

/* Readout of all runs after step n: s = sign(x), energies per replica, keep
 * the best per run (strictly lower energy replaces; k ascending). */
static void orc_eval_best(const orc_problem *pb, int P, int R, const double *x,
                          int n, int is_integer, int8_t *s, double *best_energy,
                          int32_t *best_k, int32_t *best_step, int8_t *best_s)
{
    int N = pb->n;
    size_t PN = (size_t)P * (size_t)N;
    for (int r = 0; r < R; ++r) {
        orc_sign(x + (size_t)r * PN, s, PN);
        for (int k = 0; k < P; ++k) {
            const int8_t *sk = s + (size_t)k * N;
            double e = is_integer ? (double)orc_energy_int(pb, sk) : orc_energy(pb, sk);
            if (e < best_energy[r]) {
                best_energy[r] = e;
                best_k[r] = k;
                best_step[r] = n;
                memcpy(best_s + (size_t)r * N, sk, (size_t)N);
            }
        }
    }
}

/* ------------------------------------------------------------------ */
/* Full run                                                            */
/* ------------------------------------------------------------------ */
/*
 * Runs steps [n_begin, n_end) of an S-step anneal for all R runs, starting
 * from the state in x, y (run-major, R*P*N each; the caller fills it with
 * orc_init_state for a fresh run).  beta, alpha: per-run schedule
 * parameters (Sec. II B auto-tuning draws them; here they are inputs).
 *
 * Optional outputs (NULL to skip):
 *   traj_x, traj_y   positions/momenta after each of the first n_traj steps
 *                    of the range: [(t * R * P * N) + ...]
 *   energy           R*P energies of s = sign(x) after the last step
 *   energy_int       the same as exact integers (only if is_integer)
 *   best_energy[R], best_k[R], best_step[R], best_s[R*N]
 *                    per-run best over replicas; when eval_every > 0 the
 *                    readout also runs after every step n with
 *                    (n + 1) % eval_every == 0 and keeps the best so far.
 *                    Ties: lower energy wins, then lower k, then the
 *                    earlier step (a later step must be strictly lower).
 * best_* must be initialised by the caller (best_energy = +inf) so that a
 * resumed range keeps the best found before it.
 */
void orc_run(const orc_problem *pb, const orc_params *pp, int S, int P, int R,
             const double *beta, const double *alpha, double gamma0,
             double delta_slope, int jperp_enable, int n_begin, int n_end,
             double *x, double *y, int n_traj, double *traj_x, double *traj_y,
             int eval_every, int is_integer, double *energy, int64_t *energy_int,
             double *best_energy, int32_t *best_k, int32_t *best_step,
             int8_t *best_s)
{
    int N = pb->n;
    size_t PN = (size_t)P * (size_t)N;
    double *a = (double *)malloc(sizeof(double) * (size_t)S);
    double *delta = (double *)malloc(sizeof(double) * (size_t)(S + 1));
    double *jp = (double *)malloc(sizeof(double) * (size_t)S * (size_t)R);
    int8_t *s = (int8_t *)malloc(PN);
    orc_schedule(S, P, R, gamma0, delta_slope, beta, alpha, jperp_enable, a, delta, jp);

    for (int n = n_begin; n < n_end; ++n) {
        for (int r = 0; r < R; ++r)
            orc_step_run(pb, pp, P, a[n], delta[n], jp[(size_t)r * S + n],
                         x + (size_t)r * PN, y + (size_t)r * PN);
        int t = n - n_begin;
        if (t < n_traj) {
            if (traj_x) memcpy(traj_x + (size_t)t * R * PN, x, sizeof(double) * R * PN);
            if (traj_y) memcpy(traj_y + (size_t)t * R * PN, y, sizeof(double) * R * PN);
        }
        int last = (n == n_end - 1);
        if (best_energy && (last || (eval_every > 0 && ((n + 1) % eval_every) == 0)))
            orc_eval_best(pb, P, R, x, n, is_integer, s, best_energy, best_k, best_step, best_s);
    }
    /* An empty range reads out the state it was given (step index n_begin - 1). */
    if (best_energy && n_end <= n_begin)
        orc_eval_best(pb, P, R, x, n_begin - 1, is_integer, s, best_energy, best_k, best_step, best_s);

    if (energy || energy_int) {
        for (int r = 0; r < R; ++r) {
            orc_sign(x + (size_t)r * PN, s, PN);
            for (int k = 0; k < P; ++k) {
                const int8_t *sk = s + (size_t)k * N;
                if (energy) energy[(size_t)r * P + k] = orc_energy(pb, sk);
                if (energy_int && is_integer) energy_int[(size_t)r * P + k] = orc_energy_int(pb, sk);
            }
        }
    }
    free(a);
    free(delta);
    free(jp);
    free(s);
}
