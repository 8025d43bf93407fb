/*
 * sird_oracle.h -- plain, slow FP64 CPU oracle for the SIRD-by-PSO calibration
 * method of Blaszczyk et al., "On automatic calibration of the SIRD
 * epidemiological model for COVID-19 data in Poland" (arXiv 2204.12346).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the independent reference that the
 * CUDA path is checked against.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it; the product path never does.
 * It shares no code, header, table or constant with the CUDA library.
 *
 * Everything is double precision, evaluated in the order the paper states,
 * compiled with FMA contraction off so that x86 and Arm give the same bits.
 *
 * Parity pins for every function live in tests/test_oracle_*.py.  Parity of the
 * paper's Table 1 and Figures 4-7 is unpinned: they need the paper's real data.
 */
#ifndef SIRD_ORACLE_H
#define SIRD_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Transmission-rate forms. */
enum {
    ORC_BETA_PWC = 0,  /* K equal-length constant segments over the window */
    ORC_BETA_RAMP = 1  /* the paper's eq. (beta): beta1, linear ramp, beta2 (Sec. 2.2) */
};

/* Low-level cost functions of Sec. 3.1. */
enum { ORC_MSE = 0, ORC_MXSE = 1, ORC_MAE = 2, ORC_MAPE = 3 };

/* Main objective: F_D^C (cost on D only) or F_IRD^C (max over I, R, D), Sec. 3.1. */
enum { ORC_FIT_D = 0, ORC_FIT_IRD = 1 };

/* Objectives the PSO oracle can minimise: the SIRD calibration loss, and two
 * textbook functions with known minima that pin the optimiser itself. */
enum { ORC_OBJ_SIRD = 0, ORC_OBJ_SPHERE = 1, ORC_OBJ_ROSENBROCK = 2 };

/*
 * One calibration window (Sec. 3.1): n_obs = tau+1 daily observations on days
 * 0..n_obs-1 of the window.  The initial state is S0 = N - I0 - R0 - D0 with
 * D0 = yD[0] (the Euler scheme starts from the first observation, Sec. 3.1).
 * I0 is either a fitted parameter (fit_I0 = 1, last entry of theta) or the
 * given value.  The Euler step is dt = 1/spd day, so observations fall on
 * every spd-th step.
 */
typedef struct {
    int n_obs;
    const double* yD;   /* [n_obs] cumulative deceased */
    const double* yI;   /* [n_obs] infectious, only for ORC_FIT_IRD */
    const double* yR;   /* [n_obs] recovered, only for ORC_FIT_IRD */
    double N;           /* population, constant */
    double I0;          /* initial infectious when fit_I0 == 0 */
    double R0;          /* initial recovered */
    int fit_I0;
    int beta_form;      /* ORC_BETA_PWC or ORC_BETA_RAMP */
    int K;              /* number of segments (PWC form) */
    int spd;            /* Euler steps per day, dt = 1/spd */
    int cost;           /* ORC_MSE .. ORC_MAPE */
    int objective;      /* ORC_FIT_D or ORC_FIT_IRD */
} orc_problem;

/* Number of entries of theta:
 *   PWC : (beta_1..beta_K, gamma, mu [, I0])
 *   RAMP: (beta1, beta2, t1, t2, gamma, mu [, I0])  -- t1, t2 in days from the window start */
int orc_nparams(const orc_problem* pb);

/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* Uniform in [0,1): top 24 bits of one 32-bit output times 2^-24 (exact in FP32 and FP64). */
double orc_u01(uint32_t r);

/* beta(t_k) at Euler step k (t_k = k*dt from the window start); steps_window = (n_obs-1)*spd.
 * Steps past the window keep the last segment's value (PWC) or beta2 (RAMP). */
double orc_beta(const orc_problem* pb, const double* theta, long k, long steps_window);

/* Explicit Euler on eq. (SIRD) from the window start for n_days days.
 * Writes the state at days 0..n_days (arrays of n_days+1).  Any output may be NULL.
 * Returns 0, or -1 on bad arguments. */
int orc_simulate(const orc_problem* pb, const double* theta, int n_days,
                 double* S, double* I, double* R, double* D);

/* Same, but with a per-step transmission rate beta_steps[k] (k < n_days*spd) and
 * constant gamma, mu from an explicit initial state (S0, I0, R0, D0).  Used to
 * build synthetic series with a time-varying ground truth. */
int orc_simulate_schedule(double N, double S0, double I0, double R0, double D0,
                          const double* beta_steps, double gamma, double mu,
                          int spd, int n_days,
                          double* S, double* I, double* R, double* D);

/* Calibration loss (Sec. 3.1): F_D^C or F_IRD^C of the model at theta. */
double orc_loss(const orc_problem* pb, const double* theta);

/* Coefficient of determination R^2(D) of the fitted window (Sec. 3.1). */
double orc_r2_D(const orc_problem* pb, const double* theta);

/*
 * Gradient of the discrete loss (F_D or F_IRD with MSE, MAE, MAPE or MXSE; sub-gradients
 * where the cost is not smooth, F_IRD's max through the compartment that attains it) by the
 * discrete adjoint of the Euler map.
 * g_theta[P] = dL/dtheta.  g_u0[4] = dL/d(S0, I0, R0, D0) taking the four
 * initial values as independent.  Returns the loss.
 */
double orc_loss_grad(const orc_problem* pb, const double* theta, double* g_theta, double* g_u0);

/* Deaths forecast: integrates the window and `horizon` more days with the last
 * transmission rate (beta2 / last segment), gamma and mu (Sec. 4.2); writes
 * D at days n_obs .. n_obs+horizon-1 of the window's day numbering (i.e. the
 * days after the last observed one) into D_out[horizon]. */
int orc_forecast(const orc_problem* pb, const double* theta, int horizon, double* D_out);

/* ---------------- particle swarm optimisation (Sec. 3.3) ---------------- */

typedef struct {
    int M;                 /* particles */
    int P;                 /* dimensions */
    double w, c1, c2;      /* inertia, cognitive, social */
    const double* zlb;     /* [P] bounds in search coordinates */
    const double* zub;     /* [P] */
    const int* logdim;     /* [P] 1: theta_d = exp(z_d); 0: theta_d = z_d */
    uint64_t seed;         /* Philox key */
    uint32_t stream;       /* fourth Philox counter word (window / run id) */
    int store_f32;         /* 1: swarm state and decoded theta are stored as float32 values */
    int objective_kind;    /* ORC_OBJ_* */
    uint32_t p_offset;     /* global index of particle 0: the swarm is particles p_offset ..
                              p_offset + M - 1 of a larger one (Sec. 3.3: particles are
                              independent), numbered so in the Philox counter; 0 otherwise */
} orc_pso_cfg;

/* Swarm state, particle-major: x[p*P + d]. */
typedef struct {
    double* x;        /* [M*P] positions (search coordinates) */
    double* v;        /* [M*P] velocities */
    double* pbest;    /* [M*P] personal-best positions */
    double* pbest_f;  /* [M]   personal-best values */
    double* gbest;    /* [P]   global-best position */
    int gbest_idx;
    double gbest_f;
    int iter;         /* completed PSO iterations (0 after init) */
} orc_pso_state;

/* Objective value of one search-coordinate vector z (decodes theta first). */
double orc_objective(const orc_pso_cfg* cfg, const orc_problem* pb, const double* z);

/* Draw x, v; evaluate; pbest = x; gbest = argmin. */
void orc_pso_init(const orc_pso_cfg* cfg, const orc_problem* pb, orc_pso_state* st);
/* One synchronous PSO iteration: velocity, position, clamp, evaluate, pbest, gbest. */
void orc_pso_step(const orc_pso_cfg* cfg, const orc_problem* pb, orc_pso_state* st);
/* Index of the smallest of f[0..M-1]; NaN counts as +inf; ties go to the lowest index. */
int orc_argmin(const double* f, int M);
/* Re-evaluates the k best personal bests in FP64 and returns the index of the
 * best of them by the re-evaluated value (written to *f_out). */
int orc_reeval_topk(const orc_pso_cfg* cfg, const orc_problem* pb, const orc_pso_state* st,
                    int k, double* f_out);

#ifdef __cplusplus
}
#endif

#endif
