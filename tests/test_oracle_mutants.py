"""The oracle's pins catch plausible mistakes (CPU only).

Each mutant below plants one mistake in a copy of the oracle (a dropped term, a wrong sign, a
wrong index, a swapped operand, a wrong constant), builds the copy, and runs the pins of
test_oracle_pins.py against it: at least one pin must fail.  A mutant that the pins pass would be
a part of the oracle that nothing but the oracle itself vouches for.  The real oracle is never
touched; the copies live in a temporary directory.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = os.path.join(ROOT, "tests", "test_oracle_pins.py")
C_SRC, PY_SRC = "sird_oracle.c", "__init__.py"

# (name, file, text in the oracle, planted replacement)
MUTANTS = [
    # Philox4x32-10 and the uniform conversion
    ("philox_nine_rounds", C_SRC, "round < 10; ++round", "round < 9; ++round"),
    ("philox_key_bump", C_SRC, "k1 += PHILOX_W1;", "k1 += PHILOX_W0;"),
    ("philox_swapped_multipliers", C_SRC, "mulhilo32(PHILOX_M0, c[0], &hi0, &lo0);",
     "mulhilo32(PHILOX_M1, c[0], &hi0, &lo0);"),
    ("u01_resolution", C_SRC, "(double)(r >> 8) * (1.0 / 16777216.0)", "(double)(r >> 9) * (1.0 / 8388608.0)"),
    # eq. (SIRD) and its Euler step
    ("dS_sign", C_SRC, "double fS = -beta / N * S * I;", "double fS = beta / N * S * I;"),
    ("dI_drops_mu", C_SRC, "- (gamma + mu) * I;", "- gamma * I;"),
    ("dI_transposed_operand", C_SRC, "double fI = beta / N * I * S", "double fI = beta / N * I * I"),
    ("gamma_mu_swapped", C_SRC, "double fR = gamma * I;\n    double fD = mu * I;",
     "double fR = mu * I;\n    double fD = gamma * I;"),
    ("euler_wrong_step", C_SRC, "double dt = 1.0 / (double)pb->spd;", "double dt = 1.0 / (double)(pb->spd + 1);"),
    ("S0_drops_R0", C_SRC, "u[0] = pb->N - I0 - pb->R0 - D0;", "u[0] = pb->N - I0 - D0;"),
    ("D0_not_first_observation", C_SRC, "double D0 = pb->yD[0];", "double D0 = 0.0;"),
    ("day_sampled_one_step_late", C_SRC,
     "if ((k + 1) % pb->spd == 0) put_day((int)((k + 1) / pb->spd), u, S, I, R, D);",
     "if (k % pb->spd == 0 && k > 0) put_day((int)(k / pb->spd), u, S, I, R, D);"),
    # eq. (beta)
    ("pwc_segment_off_by_one", C_SRC, "return (int)((k * (long)K) / steps_window);",
     "return (int)(((k + 1) * (long)K) / steps_window);"),
    ("pwc_segment_rounding", C_SRC, "return (int)((k * (long)K) / steps_window);",
     "return (int)((k * (long)K + steps_window / 2) / steps_window) < K ? "
     "(int)((k * (long)K + steps_window / 2) / steps_window) : K - 1;"),
    ("ramp_wrong_anchor", C_SRC, "b1 + (b2 - b1) / (t2 - t1) * (t - t1)", "b1 + (b2 - b1) / (t2 - t1) * (t - t2)"),
    ("ramp_no_ordering", C_SRC, "double t1 = theta[2] < theta[3] ? theta[2] : theta[3];",
     "double t1 = theta[2];"),
    # the costs of Sec. 3.1, F_IRD and R^2
    ("mae_wrong_mean", C_SRC, "case ORC_MAE: return acc / (double)n;",
     "case ORC_MAE: return acc / (double)(n - 1);"),
    ("mse_is_mae", C_SRC, "case ORC_MSE: acc += e * e; break;", "case ORC_MSE: acc += fabs(e); break;"),
    ("mxse_sums", C_SRC, "if (e * e > acc) acc = e * e;", "acc += e * e;"),
    ("mape_not_percent", C_SRC, "100.0 * acc / (double)kept", "acc / (double)kept"),
    ("mape_relative_to_model", C_SRC, "fabs((y[i] - yhat[i]) / y[i])", "fabs((y[i] - yhat[i]) / yhat[i])"),
    ("ird_drops_D", C_SRC, "if (cD > m) m = cD;", "(void)cD;"),
    ("ird_range_is_max", C_SRC, "return hi > lo ? hi - lo : 1.0;", "return hi > lo ? hi : 1.0;"),
    ("ird_mape_drops_I", C_SRC, "cI = low_level_cost(pb->cost, n, pb->yI, Ih, 1.0);", "cI = 0.0;"),
    ("r2_unnormalised", C_SRC, "return 1.0 - ss_res / ss_tot;", "return 1.0 - ss_res / (ss_tot + ss_res);"),
    # the discrete adjoint
    ("adjoint_beta_sign", C_SRC, "(S * I / pb->N) * (lI - lS);", "(S * I / pb->N) * (lS - lI);"),
    ("adjoint_gamma_term", C_SRC, "+= dt * I * (lR - lI);", "+= dt * I * (lD - lI);"),
    ("adjoint_state_swapped", C_SRC, "+ gamma * lR + mu * lD);", "+ gamma * lD + mu * lR);"),
    ("adjoint_drops_S_term", C_SRC, "double nI = lI + dt * (-b * S * lS + ", "double nI = lI + dt * ("),
    ("adjoint_observation_index", C_SRC, "lD += gD[k / spd];", "lD += gD[k / spd + 1];"),
    ("adjoint_ird_I_observation_index", C_SRC, "lI += gI[k / spd];", "lI += gI[k / spd + 1];"),
    ("adjoint_I0_drops_S0", C_SRC, "g_theta[idx_I0(pb)] = lI - lS;", "g_theta[idx_I0(pb)] = lI;"),
    ("adjoint_ramp_t1", C_SRC, "d_t1 = (b2 - b1) * (t - t2) / (len * len);",
     "d_t1 = (b2 - b1) * (t - t1) / (len * len);"),
    ("adjoint_mae_sign", C_SRC, "case ORC_MAE: gD[i] = -s / (double)n; break;",
     "case ORC_MAE: gD[i] = s / (double)n; break;"),
    ("adjoint_mape_percent", C_SRC, "-100.0 * s / (fabs(y[i]) * kept)", "-s / (fabs(y[i]) * kept)"),
    ("adjoint_mxse_factor", C_SRC, "(i == imax) ? -2.0 * e : 0.0", "(i == imax) ? -e : 0.0"),
    ("adjoint_ramp_b1", C_SRC, "d_b1 = 1.0 - s;", "d_b1 = s;"),
    ("adjoint_ramp_unswapped", C_SRC, "dbeta[2] = swapped ? d_t2 : d_t1;", "dbeta[2] = d_t1;"),
    ("adjoint_last_observation_dropped", C_SRC, "lD = gD[n - 1];", "lD = 0.0;"),
    ("r2_wrong_mean", C_SRC, "mean /= (double)n;", "mean /= (double)(n - 1);"),
    ("mape_counts_zero_observations", C_SRC, "if (y[i] != 0.0) { acc += fabs((y[i] - yhat[i]) / y[i]); kept++; }",
     "if (y[i] != 0.0) acc += fabs((y[i] - yhat[i]) / y[i]); kept++;"),
    ("ird_D_unnormalised", C_SRC, "cD = low_level_cost(pb->cost, n, pb->yD, Dh, series_range(n, pb->yD));",
     "cD = low_level_cost(pb->cost, n, pb->yD, Dh, 1.0);"),
    ("pwc_first_segment_after_window", C_SRC, "if (k >= steps_window) return K - 1;",
     "if (k >= steps_window) return 0;"),
    ("adjoint_beta_without_dt", C_SRC, "double dL_dbeta = dt * (S * I / pb->N)", "double dL_dbeta = (S * I / pb->N)"),
    ("adjoint_mu_term", C_SRC, "+= dt * I * (lD - lI);", "+= dt * I * (lR - lI);"),
    ("adjoint_S_sign", C_SRC, "double nS = lS + dt * (b * I * (lI - lS));", "double nS = lS + dt * (b * I * (lS - lI));"),
    ("adjoint_mse_mean", C_SRC, "case ORC_MSE: gD[i] = -2.0 * e / (double)n; break;",
     "case ORC_MSE: gD[i] = -2.0 * e / (double)(n - 1); break;"),
    ("mxse_unsquared", C_SRC, "if (e * e > acc) acc = e * e;", "if (fabs(e) > acc) acc = fabs(e);"),
    ("ird_R_range_of_I", C_SRC, "cR = low_level_cost(pb->cost, n, pb->yR, Rh, series_range(n, pb->yR));",
     "cR = low_level_cost(pb->cost, n, pb->yR, Rh, series_range(n, pb->yI));"),
    ("ramp_right_endpoint", C_SRC, "double t = (double)k / (double)pb->spd;\n    if (t < t1) return b1;",
     "double t = (double)(k + 1) / (double)pb->spd;\n    if (t < t1) return b1;"),
    ("pwc_past_window_boundary", C_SRC, "if (k >= steps_window) return K - 1;", "if (k > steps_window) return K - 1;"),
    ("fixed_I0_ignored", C_SRC, "double I0 = pb->fit_I0 ? theta[idx_I0(pb)] : pb->I0;", "double I0 = pb->fit_I0 ? theta[idx_I0(pb)] : 0.0;"),
    ("window_one_day_long", C_SRC, "long steps_window = (long)(pb->n_obs - 1) * pb->spd;",
     "long steps_window = (long)pb->n_obs * pb->spd;"),
    ("ramp_after_t2_is_beta1", C_SRC, "    return b2;\n}", "    return b1;\n}"),
    ("r2_total_unsquared", C_SRC, "ss_tot += (pb->yD[i] - mean) * (pb->yD[i] - mean);", "ss_tot += fabs(pb->yD[i] - mean);"),
    ("schedule_rate_one_step_late", C_SRC, "euler_step(N, beta_steps[k], gamma, mu, dt, u);",
     "euler_step(N, beta_steps[k > 0 ? k - 1 : 0], gamma, mu, dt, u);"),
    # the forecast of Sec. 4.2
    ("forecast_repeats_last_day", C_SRC, "D_out[h] = D[L + 1 + h];", "D_out[h] = D[L + h];"),
    # the PSO of Sec. 3.3
    ("pso_cognitive_sign", C_SRC, "cfg->c1 * r1 * (pb_x[d] - x[d])", "cfg->c1 * r1 * (x[d] - pb_x[d])"),
    ("pso_social_operand", C_SRC, "cfg->c2 * r2 * (st->gbest[d] - x[d])", "cfg->c2 * r2 * (st->gbest[d] - pb_x[d])"),
    ("pso_inertia_on_position", C_SRC, "cfg->w * v[d]", "cfg->w * x[d]"),
    ("pso_same_random_number", C_SRC, "cfg->c2 * r2 *", "cfg->c2 * r1 *"),
    ("pso_no_upper_clamp", C_SRC, "if (xn > cfg->zub[d]) xn = cfg->zub[d];", ""),
    ("pso_velocity_zeroed_at_bound", C_SRC, "v[d] = vn;",
     "v[d] = (xn == cfg->zlb[d] || xn == cfg->zub[d]) ? 0.0 : vn;"),
    ("pso_pbest_always_replaced", C_SRC, "if (f < st->pbest_f[p]) {", "if (f == f) {"),
    ("pso_init_velocity_one_sided", C_SRC, "range * (2.0 * ub - 1.0)", "range * ub"),
    ("pso_log_box_not_decoded", C_SRC, "cfg->logdim && cfg->logdim[d] ? exp(z[d]) : z[d]", "z[d]"),
    ("argmin_last_of_ties", C_SRC, "if (v < bf) { bf = v; best = p; }", "if (v <= bf) { bf = v; best = p; }"),
    ("argmin_nan_first", C_SRC, "double bf = isnan(f[0]) ? INFINITY : f[0];", "double bf = f[0];"),
    ("reeval_in_search_precision", C_SRC, "c64.store_f32 = 0;", "c64.store_f32 = cfg->store_f32;"),
    ("reeval_first_of_k_only", C_SRC, "for (int j = 0; j < k; ++j) {", "for (int j = 0; j < 1; ++j) {"),
    ("pso_position_with_old_velocity", C_SRC, "double xn = store(cfg, x[d] + vn);", "double xn = store(cfg, x[d] + v[d]);"),
    ("pso_no_lower_clamp", C_SRC, "if (xn < cfg->zlb[d]) xn = cfg->zlb[d];", ""),
    ("gbest_from_positions", C_SRC, "memcpy(st->gbest, st->pbest + (size_t)g * cfg->P, sizeof(double) * cfg->P);",
     "memcpy(st->gbest, st->x + (size_t)g * cfg->P, sizeof(double) * cfg->P);"),
    ("pbest_position_not_copied", C_SRC, "memcpy(st->pbest + (size_t)p * P, x, sizeof(double) * P);", ""),
    ("nan_loss_not_infinite", C_SRC, "return isnan(f) ? INFINITY : f;", "return f;"),
    ("pso_particle_offset_ignored", C_SRC, "(uint32_t)p + cfg->p_offset", "(uint32_t)p"),
    ("store_f32_ignored", C_SRC, "return cfg->store_f32 ? (double)(float)x : x;", "return x;"),
    # the F_IRD^C gradient
    ("ird_grad_drops_R_injection", C_SRC, "lR += gR[k / spd];", "(void)0;"),
    ("ird_grad_I_unscaled", C_SRC, "cost_grad_series(pb->cost, n, pb->yI, Ih, sI, gI)",
     "cost_grad_series(pb->cost, n, pb->yI, Ih, 1.0, gI)"),
    ("ird_grad_mxse_unscaled", C_SRC, "-2.0 * e / scale : 0.0", "-2.0 * e : 0.0"),
    ("ird_grad_mse_scaled_once", C_SRC, "-2.0 * e / ((double)n * scale)", "-2.0 * e / (double)n"),
    ("ird_grad_last_day_of_I", C_SRC, "lI = gI[n - 1]", "lI = 0.0"),
    ("ird_grad_never_I", C_SRC, "if (which == 0) cost_grad_series", "if (0) cost_grad_series"),
    ("ird_grad_mae_sign", C_SRC, "case ORC_MAE: g[i] = -s / ((double)n * scale); break;",
     "case ORC_MAE: g[i] = s / ((double)n * scale); break;"),
    # the ensemble bands of Sec. 4.2
    ("bands_median_upper_middle", PY_SRC, "(v[:, k // 2 - 1] + v[:, k // 2]) * 0.5", "v[:, k // 2]"),
    ("bands_R0_drops_mu", PY_SRC, "beta / (th[j, gi] + th[j, gi + 1])", "beta / th[j, gi]"),
    ("bands_drop_both_tails", PY_SRC, "k * (1.0 - f) / 2.0", "k * (1.0 - f)"),
    ("bands_beta_one_step_late", PY_SRC, "beta_at(pb, th[j], d * pb.spd)", "beta_at(pb, th[j], d * pb.spd + 1)"),
    ("bands_low_index", PY_SRC, "cols += [v[:, dr], v[:, k - 1 - dr]]", "cols += [v[:, min(dr + 1, k - 1)], v[:, k - 1 - dr]]"),
    ("bands_gamma_index", PY_SRC, "gi = 4 if pb.beta_form == BETA_RAMP else pb.K", "gi = 4 if pb.beta_form == BETA_RAMP else pb.K - 1"),
    ("bands_high_index", PY_SRC, "v[:, k - 1 - dr]", "v[:, k - dr - 2 if k - dr - 2 >= 0 else 0]"),
    # the parameter bands of Sec. 4.2
    ("pbands_median_upper_middle", PY_SRC, "(v[k // 2 - 1] + v[k // 2]) * 0.5", "v[k // 2]"),
    ("pbands_low_index", PY_SRC, "out[d, 1 + 2 * b] = v[dr]", "out[d, 1 + 2 * b] = v[min(dr + 1, k - 1)]"),
    ("pbands_high_index", PY_SRC, "out[d, 2 + 2 * b] = v[k - 1 - dr]", "out[d, 2 + 2 * b] = v[max(k - 2 - dr, 0)]"),
    ("pbands_ramp_times_unordered", PY_SRC, "th[:, 2] = np.minimum(ta, tb)", "th[:, 2] = ta"),
    ("pbands_ramp_end_unordered", PY_SRC, "th[:, 3] = np.maximum(ta, tb)", "th[:, 3] = tb"),
]


def _run_pins_on(name, fname, old, new, workdir, extra_env=None, extra_args=()):
    src_dir = os.path.join(ROOT, "oracle")
    dst = os.path.join(workdir, name)
    pkg = os.path.join(dst, "oracle")
    os.makedirs(pkg)
    for f in ("sird_oracle.c", "sird_oracle.h", "__init__.py"):
        shutil.copy(os.path.join(src_dir, f), os.path.join(pkg, f))
    path = os.path.join(pkg, fname)
    text = open(path).read()
    assert text.count(old) == 1, f"{name}: the mutated text must occur exactly once in {fname}"
    open(path, "w").write(text.replace(old, new))
    env = dict(os.environ, PYTHONPATH=os.pathsep.join([dst, ROOT]), PYTHONDONTWRITEBYTECODE="1", **(extra_env or {}))
    # cwd = the copy, so that `import oracle` finds the mutant first
    r = subprocess.run([sys.executable, "-m", "pytest", PINS, "-x", "-q", "-p", "no:cacheprovider", *extra_args],
                       cwd=dst, env=env, capture_output=True, text=True, timeout=600)
    return name, r.returncode, r.stdout[-2000:] + r.stderr[-2000:]


@pytest.fixture(scope="module")
def mutant_runs(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    work = str(tmp_path_factory.mktemp("mutants"))
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        runs = list(ex.map(lambda m: _run_pins_on(*m, work), MUTANTS))
    return {name: (rc, out) for name, rc, out in runs}


def test_mutant_names_are_unique():
    assert len({m[0] for m in MUTANTS}) == len(MUTANTS)


def test_the_unmutated_copy_passes_the_pins(tmp_path):
    # the harness itself: a copy with a no-op change passes, so a failing mutant fails for its mistake
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    _, rc, out = _run_pins_on("identity", C_SRC, "#include <math.h>", "#include <math.h>", str(tmp_path))
    assert rc == 0, out


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS])
def test_pins_catch_the_mutant(mutant_runs, name):
    rc, out = mutant_runs[name]
    # 1: tests ran and at least one failed (not a build or collection error); a mutant that
    # crashes the pins (killed by a signal) is caught as well
    assert rc == 1 or rc < 0, f"mutant {name} survived the pins (exit {rc}):\n{out}"


def test_pins_pass_with_the_oracle_under_address_and_undefined_behaviour_sanitizers(tmp_path):
    # the oracle built with ASan + UBSan (aborting on the first report) runs every pin cleanly:
    # no out-of-bounds access, use after free, signed overflow or out-of-range float conversion
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    asan = subprocess.run([gcc, "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    if not os.path.isabs(asan) or not os.path.exists(asan):
        pytest.skip("no ASan runtime")
    flags = '"-fsanitize=address,undefined,float-cast-overflow", "-fno-sanitize-recover=all", "-o", tmp'
    # -s: pytest leaves stderr alone, so a sanitizer's report reaches the output checked here
    _, rc, out = _run_pins_on("sanitized", PY_SRC, '"-o", tmp', flags, str(tmp_path),
                              extra_env={"LD_PRELOAD": asan, "ASAN_OPTIONS": "detect_leaks=0"}, extra_args=("-s",))
    assert rc == 0, out
    assert "runtime error" not in out and "AddressSanitizer" not in out, out
