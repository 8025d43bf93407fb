/*
 * sird_oracle.c -- plain, slow FP64 CPU oracle (test infrastructure only).
 *
 * Written from the paper (arXiv 2204.12346):
 *   Sec. 2.2, eq. (SIRD)  the model S' = -beta S I / N, I' = beta I S / N - (gamma+mu) I,
 *                         R' = gamma I, D' = mu I
 *   Sec. 2.2, eq. (beta)  the time-varying transmission rate (ramp form)
 *   Sec. 3.1              windows, explicit Euler from the first observation,
 *                         the costs MXSE / MSE / MAE / MAPE, F_D^C, F_IRD^C, R^2(D)
 *   Sec. 3.3              particle swarm optimisation, out-of-bounds values set to the bound
 *   Sec. 4.2              the extension of a fitted window with (beta2, gamma, mu)
 * plus Philox4x32-10 from Salmon, Moraes, Dror and Shaw, "Parallel random numbers:
 * as easy as 1, 2, 3" (SC'11).
 *
 * The state is carried as the paper writes it (S, I, R, D), in double precision,
 * one Euler step at a time.  No blocking, fusion or reordering.
 */
#include "sird_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ Philox */

/* Round multipliers and Weyl key increments as published for Philox4x32. */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

static void mulhilo32(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo) {
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { /* the key is bumped before every round but the first */
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint32_t hi0, lo0, hi1, lo1;
        mulhilo32(PHILOX_M0, c[0], &hi0, &lo0);
        mulhilo32(PHILOX_M1, c[2], &hi1, &lo1);
        uint32_t n0 = hi1 ^ c[1] ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c[3] ^ k1;
        uint32_t n3 = lo0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

double orc_u01(uint32_t r) { return (double)(r >> 8) * (1.0 / 16777216.0); }

/* ------------------------------------------------------------------ model */

int orc_nparams(const orc_problem* pb) {
    int base = (pb->beta_form == ORC_BETA_RAMP) ? 6 : pb->K + 2;
    return base + (pb->fit_I0 ? 1 : 0);
}

static int idx_gamma(const orc_problem* pb) { return pb->beta_form == ORC_BETA_RAMP ? 4 : pb->K; }
static int idx_mu(const orc_problem* pb) { return idx_gamma(pb) + 1; }
static int idx_I0(const orc_problem* pb) { return idx_gamma(pb) + 2; }

/* PWC segment of step k: floor(k*K/steps) for k inside the window, last segment after it. */
static int pwc_segment(long k, long steps_window, int K) {
    if (k >= steps_window) return K - 1;
    return (int)((k * (long)K) / steps_window);
}

double orc_beta(const orc_problem* pb, const double* theta, long k, long steps_window) {
    if (pb->beta_form == ORC_BETA_PWC) return theta[pwc_segment(k, steps_window, pb->K)];
    /* eq. (beta): beta1 on [a, t1), linear from beta1 to beta2 on [t1, t2), beta2 from t2 on.
     * The search box cannot enforce t1 <= t2, so the smaller of the two is taken as t1. */
    double b1 = theta[0], b2 = theta[1];
    double t1 = theta[2] < theta[3] ? theta[2] : theta[3];
    double t2 = theta[2] < theta[3] ? theta[3] : theta[2];
    double t = (double)k / (double)pb->spd;
    if (t < t1) return b1;
    if (t < t2) return b1 + (b2 - b1) / (t2 - t1) * (t - t1);
    return b2;
}

static void initial_state(const orc_problem* pb, const double* theta, double u[4]) {
    double I0 = pb->fit_I0 ? theta[idx_I0(pb)] : pb->I0;
    double D0 = pb->yD[0]; /* Euler starts from the first observation */
    u[1] = I0;
    u[2] = pb->R0;
    u[3] = D0;
    u[0] = pb->N - I0 - pb->R0 - D0;
}

/* One explicit Euler step of eq. (SIRD) with rates beta, gamma, mu. */
static void euler_step(double N, double beta, double gamma, double mu, double dt, double u[4]) {
    double S = u[0], I = u[1];
    double fS = -beta / N * S * I;
    double fI = beta / N * I * S - (gamma + mu) * I;
    double fR = gamma * I;
    double fD = mu * I;
    u[0] = S + dt * fS;
    u[1] = I + dt * fI;
    u[2] = u[2] + dt * fR;
    u[3] = u[3] + dt * fD;
}

static void put_day(int day, const double u[4], double* S, double* I, double* R, double* D) {
    if (S) S[day] = u[0];
    if (I) I[day] = u[1];
    if (R) R[day] = u[2];
    if (D) D[day] = u[3];
}

int orc_simulate(const orc_problem* pb, const double* theta, int n_days,
                 double* S, double* I, double* R, double* D) {
    if (!pb || !theta || n_days < 0 || pb->spd < 1 || pb->n_obs < 1) return -1;
    if (pb->beta_form == ORC_BETA_PWC && pb->K < 1) return -1;
    double u[4];
    initial_state(pb, theta, u);
    double gamma = theta[idx_gamma(pb)], mu = theta[idx_mu(pb)];
    double dt = 1.0 / (double)pb->spd;
    long steps_window = (long)(pb->n_obs - 1) * pb->spd;
    long steps = (long)n_days * pb->spd;
    put_day(0, u, S, I, R, D);
    for (long k = 0; k < steps; ++k) {
        double beta = orc_beta(pb, theta, k, steps_window);
        euler_step(pb->N, beta, gamma, mu, dt, u);
        if ((k + 1) % pb->spd == 0) put_day((int)((k + 1) / pb->spd), u, S, I, R, D);
    }
    return 0;
}

int orc_simulate_schedule(double N, double S0, double I0, double R0, double D0,
                          const double* beta_steps, double gamma, double mu,
                          int spd, int n_days,
                          double* S, double* I, double* R, double* D) {
    if (!beta_steps || spd < 1 || n_days < 0) return -1;
    double u[4] = {S0, I0, R0, D0};
    double dt = 1.0 / (double)spd;
    put_day(0, u, S, I, R, D);
    for (long k = 0; k < (long)n_days * spd; ++k) {
        euler_step(N, beta_steps[k], gamma, mu, dt, u);
        if ((k + 1) % spd == 0) put_day((int)((k + 1) / spd), u, S, I, R, D);
    }
    return 0;
}

/* ------------------------------------------------------------------ costs */

/* Low-level cost C over n errors e_i = y_i - yhat_i (Sec. 3.1).  For MAPE the
 * relative errors use y_i; terms with y_i == 0 are skipped and the mean is taken
 * over the terms kept (the paper does not say what to do with y_i == 0). */
static double low_level_cost(int cost, int n, const double* y, const double* yhat, double scale) {
    double acc = 0.0;
    int kept = 0;
    for (int i = 0; i < n; ++i) {
        double e = (y[i] - yhat[i]) / scale;
        switch (cost) {
            case ORC_MSE: acc += e * e; break;
            case ORC_MXSE: if (e * e > acc) acc = e * e; break;
            case ORC_MAE: acc += fabs(e); break;
            case ORC_MAPE:
                if (y[i] != 0.0) { acc += fabs((y[i] - yhat[i]) / y[i]); kept++; }
                break;
            default: return NAN;
        }
    }
    switch (cost) {
        case ORC_MSE:
        case ORC_MAE: return acc / (double)n;
        case ORC_MXSE: return acc;
        default: return kept > 0 ? 100.0 * acc / (double)kept : 0.0;
    }
}

/* Range of the reported series used by the min-max normalisation f_Y (Sec. 3.1).
 * A flat series (max == min) is left unscaled. */
static double series_range(int n, const double* y) {
    double lo = y[0], hi = y[0];
    for (int i = 1; i < n; ++i) {
        if (y[i] < lo) lo = y[i];
        if (y[i] > hi) hi = y[i];
    }
    return hi > lo ? hi - lo : 1.0;
}

static double loss_from_days(const orc_problem* pb, const double* Ih, const double* Rh, const double* Dh) {
    int n = pb->n_obs;
    if (pb->objective == ORC_FIT_D) return low_level_cost(pb->cost, n, pb->yD, Dh, 1.0);
    /* F_IRD: max over the three compartments.  f_Y(y) - f_Y(yhat) = (y - yhat)/(max - min),
     * so the min-max normalisation divides each error by the reported range;
     * MAPE is taken without normalisation. */
    double cI, cR, cD;
    if (pb->cost == ORC_MAPE) {
        cI = low_level_cost(pb->cost, n, pb->yI, Ih, 1.0);
        cR = low_level_cost(pb->cost, n, pb->yR, Rh, 1.0);
        cD = low_level_cost(pb->cost, n, pb->yD, Dh, 1.0);
    } else {
        cI = low_level_cost(pb->cost, n, pb->yI, Ih, series_range(n, pb->yI));
        cR = low_level_cost(pb->cost, n, pb->yR, Rh, series_range(n, pb->yR));
        cD = low_level_cost(pb->cost, n, pb->yD, Dh, series_range(n, pb->yD));
    }
    double m = cI;
    if (cR > m) m = cR;
    if (cD > m) m = cD;
    return m;
}

double orc_loss(const orc_problem* pb, const double* theta) {
    int n = pb->n_obs;
    double* I = (double*)malloc(sizeof(double) * n);
    double* R = (double*)malloc(sizeof(double) * n);
    double* D = (double*)malloc(sizeof(double) * n);
    double L = NAN;
    if (I && R && D && orc_simulate(pb, theta, n - 1, NULL, I, R, D) == 0) L = loss_from_days(pb, I, R, D);
    free(I); free(R); free(D);
    return L;
}

double orc_r2_D(const orc_problem* pb, const double* theta) {
    int n = pb->n_obs;
    double* D = (double*)malloc(sizeof(double) * n);
    if (!D || orc_simulate(pb, theta, n - 1, NULL, NULL, NULL, D) != 0) { free(D); return NAN; }
    double mean = 0.0;
    for (int i = 0; i < n; ++i) mean += pb->yD[i];
    mean /= (double)n;
    double ss_res = 0.0, ss_tot = 0.0;
    for (int i = 0; i < n; ++i) {
        double e = pb->yD[i] - D[i];
        ss_res += e * e;
        ss_tot += (pb->yD[i] - mean) * (pb->yD[i] - mean);
    }
    free(D);
    return 1.0 - ss_res / ss_tot;
}

/* ------------------------------------------------------------------ adjoint */

/* dL/dDhat_i for the F_D costs (sub-gradients where the cost is not smooth). */
static void cost_grad_D(const orc_problem* pb, const double* Dh, double* gD) {
    int n = pb->n_obs;
    const double* y = pb->yD;
    int kept = 0, imax = 0;
    double emax = -1.0;
    for (int i = 0; i < n; ++i) {
        if (y[i] != 0.0) kept++;
        double e = y[i] - Dh[i];
        if (e * e > emax) { emax = e * e; imax = i; }
    }
    for (int i = 0; i < n; ++i) {
        double e = y[i] - Dh[i];
        double s = (e > 0.0) - (e < 0.0);
        switch (pb->cost) {
            case ORC_MSE: gD[i] = -2.0 * e / (double)n; break;
            case ORC_MAE: gD[i] = -s / (double)n; break;
            case ORC_MAPE: gD[i] = (y[i] != 0.0 && kept > 0) ? -100.0 * s / (fabs(y[i]) * kept) : 0.0; break;
            case ORC_MXSE: gD[i] = (i == imax) ? -2.0 * e : 0.0; break;
            default: gD[i] = NAN;
        }
    }
}

/* dC/dyhat_i of one series' low-level cost C (as low_level_cost computes it) over the errors
 * e_i = (y_i - yhat_i) / scale: MSE -2 e_i / (n scale), MAE -sign(e_i) / (n scale), MXSE
 * -2 e_i / scale at the first day with the largest e^2 (none when every e is 0), MAPE
 * -100 sign(y_i - yhat_i) / (|y_i| kept) on the days with y_i != 0. */
static void cost_grad_series(int cost, int n, const double* y, const double* yhat, double scale, double* g) {
    int kept = 0, imax = -1;
    double acc = 0.0;
    for (int i = 0; i < n; ++i) {
        if (y[i] != 0.0) kept++;
        double e = (y[i] - yhat[i]) / scale;
        if (e * e > acc) { acc = e * e; imax = i; }
    }
    for (int i = 0; i < n; ++i) {
        double e = (y[i] - yhat[i]) / scale;
        double s = (e > 0.0) - (e < 0.0);
        switch (cost) {
            case ORC_MSE: g[i] = -2.0 * e / ((double)n * scale); break;
            case ORC_MAE: g[i] = -s / ((double)n * scale); break;
            case ORC_MAPE: g[i] = (y[i] != 0.0 && kept > 0) ? -100.0 * s / (fabs(y[i]) * (double)kept) : 0.0; break;
            case ORC_MXSE: g[i] = (i == imax) ? -2.0 * e / scale : 0.0; break;
            default: g[i] = NAN;
        }
    }
}

/* d beta(t_k) / d theta for the ramp form (only the four beta-form entries). */
static void ramp_dbeta(const orc_problem* pb, const double* theta, long k, double dbeta[4]) {
    double b1 = theta[0], b2 = theta[1];
    int swapped = theta[2] > theta[3];
    double t1 = swapped ? theta[3] : theta[2];
    double t2 = swapped ? theta[2] : theta[3];
    double t = (double)k / (double)pb->spd;
    double d_b1 = 0, d_b2 = 0, d_t1 = 0, d_t2 = 0;
    if (t < t1) {
        d_b1 = 1.0;
    } else if (t < t2) {
        double len = t2 - t1, s = (t - t1) / len;
        d_b1 = 1.0 - s;
        d_b2 = s;
        d_t1 = (b2 - b1) * (t - t2) / (len * len);
        d_t2 = -(b2 - b1) * (t - t1) / (len * len);
    } else {
        d_b2 = 1.0;
    }
    dbeta[0] = d_b1;
    dbeta[1] = d_b2;
    dbeta[2] = swapped ? d_t2 : d_t1;
    dbeta[3] = swapped ? d_t1 : d_t2;
}

double orc_loss_grad(const orc_problem* pb, const double* theta, double* g_theta, double* g_u0) {
    int n = pb->n_obs, spd = pb->spd, P = orc_nparams(pb);
    long steps = (long)(n - 1) * spd;
    double dt = 1.0 / (double)spd;
    double gamma = theta[idx_gamma(pb)], mu = theta[idx_mu(pb)];
    double* U = (double*)malloc(sizeof(double) * 4 * (size_t)(steps + 1));
    double* Yh = (double*)malloc(sizeof(double) * 3 * (size_t)n);   /* Ihat | Rhat | Dhat per day */
    double* gY = (double*)calloc(3 * (size_t)n, sizeof(double));    /* dL/dIhat | dL/dRhat | dL/dDhat */
    if (!U || !Yh || !gY) { free(U); free(Yh); free(gY); return NAN; }
    double *Ih = Yh, *Rh = Yh + n, *Dh = Yh + 2 * n;
    double *gI = gY, *gR = gY + n, *gD = gY + 2 * n;

    /* forward sweep, keeping every state */
    initial_state(pb, theta, U);
    for (long k = 0; k < steps; ++k) {
        memcpy(U + 4 * (k + 1), U + 4 * k, 4 * sizeof(double));
        euler_step(pb->N, orc_beta(pb, theta, k, steps), gamma, mu, dt, U + 4 * (k + 1));
    }
    for (int i = 0; i < n; ++i) {
        Ih[i] = U[4 * ((long)i * spd) + 1];
        Rh[i] = U[4 * ((long)i * spd) + 2];
        Dh[i] = U[4 * ((long)i * spd) + 3];
    }
    double L;
    if (pb->objective == ORC_FIT_D) {
        L = low_level_cost(pb->cost, n, pb->yD, Dh, 1.0);
        cost_grad_D(pb, Dh, gD);
    } else {
        /* F_IRD^C = max(C_I, C_R, C_D) (Sec. 3.1): the gradient of the compartment that attains
         * the maximum (the first of I, R, D on ties), as loss_from_days picks it; each error
         * divided by its reported range, MAPE unnormalised. */
        int mape = pb->cost == ORC_MAPE;
        double sI = mape ? 1.0 : series_range(n, pb->yI);
        double sR = mape ? 1.0 : series_range(n, pb->yR);
        double sD = mape ? 1.0 : series_range(n, pb->yD);
        double cI = low_level_cost(pb->cost, n, pb->yI, Ih, sI);
        double cR = low_level_cost(pb->cost, n, pb->yR, Rh, sR);
        double cD = low_level_cost(pb->cost, n, pb->yD, Dh, sD);
        int which = 0;
        L = cI;
        if (cR > L) { L = cR; which = 1; }
        if (cD > L) { L = cD; which = 2; }
        if (which == 0) cost_grad_series(pb->cost, n, pb->yI, Ih, sI, gI);
        else if (which == 1) cost_grad_series(pb->cost, n, pb->yR, Rh, sR, gR);
        else cost_grad_series(pb->cost, n, pb->yD, Dh, sD, gD);
    }

    /* reverse sweep: lambda_k = lambda_{k+1} + dt (df/du)^T lambda_{k+1} + dL/du_k */
    for (int j = 0; j < P; ++j) g_theta[j] = 0.0;
    double lS = 0.0, lI = gI[n - 1], lR = gR[n - 1], lD = gD[n - 1];
    for (long k = steps - 1; k >= 0; --k) {
        const double* u = U + 4 * k;
        double S = u[0], I = u[1];
        double beta = orc_beta(pb, theta, k, steps);
        double b = beta / pb->N;
        /* parameter gradients use lambda_{k+1} */
        double dL_dbeta = dt * (S * I / pb->N) * (lI - lS);
        if (pb->beta_form == ORC_BETA_PWC) {
            g_theta[pwc_segment(k, steps, pb->K)] += dL_dbeta;
        } else {
            double db[4];
            ramp_dbeta(pb, theta, k, db);
            for (int j = 0; j < 4; ++j) g_theta[j] += dL_dbeta * db[j];
        }
        g_theta[idx_gamma(pb)] += dt * I * (lR - lI);
        g_theta[idx_mu(pb)] += dt * I * (lD - lI);
        /* state adjoint */
        double nS = lS + dt * (b * I * (lI - lS));
        double nI = lI + dt * (-b * S * lS + (b * S - gamma - mu) * lI + gamma * lR + mu * lD);
        lS = nS;
        lI = nI;
        if (k % spd == 0) {
            lI += gI[k / spd];
            lR += gR[k / spd];
            lD += gD[k / spd];
        }
    }
    if (pb->fit_I0) g_theta[idx_I0(pb)] = lI - lS; /* S0 = N - I0 - R0 - D0 */
    if (g_u0) { g_u0[0] = lS; g_u0[1] = lI; g_u0[2] = lR; g_u0[3] = lD; }
    free(U); free(Yh); free(gY);
    return L;
}

/* ------------------------------------------------------------------ forecast */

int orc_forecast(const orc_problem* pb, const double* theta, int horizon, double* D_out) {
    if (horizon < 0) return -1;
    int L = pb->n_obs - 1;
    double* D = (double*)malloc(sizeof(double) * (size_t)(L + horizon + 1));
    if (!D) return -1;
    int rc = orc_simulate(pb, theta, L + horizon, NULL, NULL, NULL, D);
    if (rc == 0) for (int h = 0; h < horizon; ++h) D_out[h] = D[L + 1 + h];
    free(D);
    return rc;
}

/* ------------------------------------------------------------------ PSO */

static double store(const orc_pso_cfg* cfg, double x) { return cfg->store_f32 ? (double)(float)x : x; }

static double eval_theta(const orc_pso_cfg* cfg, const orc_problem* pb, const double* th) {
    int P = cfg->P;
    double f;
    switch (cfg->objective_kind) {
        case ORC_OBJ_SIRD: f = orc_loss(pb, th); break;
        case ORC_OBJ_SPHERE:
            f = 0.0;
            for (int d = 0; d < P; ++d) f += th[d] * th[d];
            break;
        case ORC_OBJ_ROSENBROCK:
            f = 0.0;
            for (int d = 0; d + 1 < P; ++d)
                f += 100.0 * (th[d + 1] - th[d] * th[d]) * (th[d + 1] - th[d] * th[d]) + (1.0 - th[d]) * (1.0 - th[d]);
            break;
        default: f = NAN;
    }
    return isnan(f) ? INFINITY : f;
}

double orc_objective(const orc_pso_cfg* cfg, const orc_problem* pb, const double* z) {
    double th[64];
    for (int d = 0; d < cfg->P; ++d) th[d] = store(cfg, cfg->logdim && cfg->logdim[d] ? exp(z[d]) : z[d]);
    return eval_theta(cfg, pb, th);
}

int orc_argmin(const double* f, int M) {
    int best = 0;
    double bf = isnan(f[0]) ? INFINITY : f[0];
    for (int p = 1; p < M; ++p) {
        double v = isnan(f[p]) ? INFINITY : f[p];
        if (v < bf) { bf = v; best = p; }
    }
    return best;
}

static void set_gbest(const orc_pso_cfg* cfg, orc_pso_state* st) {
    int g = orc_argmin(st->pbest_f, cfg->M);
    st->gbest_idx = g;
    st->gbest_f = st->pbest_f[g];
    memcpy(st->gbest, st->pbest + (size_t)g * cfg->P, sizeof(double) * cfg->P);
}

/* Philox counter layout: (particle, iteration, dimension pair, stream word).  One
 * call gives four words; dimension d uses words 2*(d%2) and 2*(d%2)+1 as its (r1, r2)
 * (at iteration 0: the position and velocity draws). */
static void draw(const orc_pso_cfg* cfg, int p, int d, int iter, double* u_a, double* u_b) {
    uint32_t ctr[4] = {(uint32_t)p + cfg->p_offset, (uint32_t)iter, (uint32_t)(d >> 1), cfg->stream};
    uint32_t key[2] = {(uint32_t)cfg->seed, (uint32_t)(cfg->seed >> 32)};
    uint32_t r[4];
    orc_philox4x32_10(ctr, key, r);
    *u_a = orc_u01(r[2 * (d & 1)]);
    *u_b = orc_u01(r[2 * (d & 1) + 1]);
}

void orc_pso_init(const orc_pso_cfg* cfg, const orc_problem* pb, orc_pso_state* st) {
    int M = cfg->M, P = cfg->P;
    for (int p = 0; p < M; ++p) {
        for (int d = 0; d < P; ++d) {
            double ua, ub;
            draw(cfg, p, d, 0, &ua, &ub);
            double range = cfg->zub[d] - cfg->zlb[d];
            double x = store(cfg, cfg->zlb[d] + range * ua);
            if (x > cfg->zub[d]) x = cfg->zub[d];
            st->x[(size_t)p * P + d] = x;
            st->v[(size_t)p * P + d] = store(cfg, range * (2.0 * ub - 1.0));
        }
        st->pbest_f[p] = store(cfg, orc_objective(cfg, pb, st->x + (size_t)p * P));
    }
    memcpy(st->pbest, st->x, sizeof(double) * (size_t)M * P);
    st->iter = 0;
    set_gbest(cfg, st);
}

void orc_pso_step(const orc_pso_cfg* cfg, const orc_problem* pb, orc_pso_state* st) {
    int M = cfg->M, P = cfg->P, t = st->iter + 1;
    for (int p = 0; p < M; ++p) {
        double* x = st->x + (size_t)p * P;
        double* v = st->v + (size_t)p * P;
        const double* pb_x = st->pbest + (size_t)p * P;
        for (int d = 0; d < P; ++d) {
            double r1, r2;
            draw(cfg, p, d, t, &r1, &r2);
            double vn = store(cfg, cfg->w * v[d] + cfg->c1 * r1 * (pb_x[d] - x[d]) + cfg->c2 * r2 * (st->gbest[d] - x[d]));
            double xn = store(cfg, x[d] + vn);
            /* out-of-bounds values are set to the bound (Sec. 3.3); the velocity is kept */
            if (xn < cfg->zlb[d]) xn = cfg->zlb[d];
            if (xn > cfg->zub[d]) xn = cfg->zub[d];
            v[d] = vn;
            x[d] = xn;
        }
        double f = store(cfg, orc_objective(cfg, pb, x));
        if (f < st->pbest_f[p]) {
            st->pbest_f[p] = f;
            memcpy(st->pbest + (size_t)p * P, x, sizeof(double) * P);
        }
    }
    st->iter = t;
    set_gbest(cfg, st);
}

int orc_reeval_topk(const orc_pso_cfg* cfg, const orc_problem* pb, const orc_pso_state* st,
                    int k, double* f_out) {
    int M = cfg->M, P = cfg->P;
    if (k > M) k = M;
    if (k < 1) k = 1;
    char* taken = (char*)calloc((size_t)M, 1);
    int best = -1;
    double best_f = INFINITY;
    orc_pso_cfg c64 = *cfg;
    c64.store_f32 = 0; /* the re-evaluation decodes and evaluates in FP64 */
    for (int j = 0; j < k; ++j) {
        /* j-th smallest personal best, lowest index first among equals */
        int pick = -1;
        double pf = INFINITY;
        for (int p = 0; p < M; ++p) {
            if (taken[p]) continue;
            double v = isnan(st->pbest_f[p]) ? INFINITY : st->pbest_f[p];
            if (pick < 0 || v < pf) { pick = p; pf = v; }
        }
        taken[pick] = 1;
        double f = orc_objective(&c64, pb, st->pbest + (size_t)pick * P);
        if (best < 0 || f < best_f || (f == best_f && pick < best)) { best = pick; best_f = f; }
    }
    free(taken);
    if (f_out) *f_out = best_f;
    return best;
}
