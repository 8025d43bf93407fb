"""The C-ABI library builds for sm_103a, loads, exports what the header declares, and
rejects bad arguments before touching the GPU (CPU only)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2204_12346_gb300 import build, sird

    build.build()
    return sird.lib()


def test_header_and_exports_agree(L):
    from paper_2204_12346_gb300 import sird

    header = open(os.path.join(ROOT, "include", "sird_pso.h")).read()
    header = re.sub(r"/\*.*?\*/", "", header, flags=re.S)
    declared = set(re.findall(r"\b(sird_\w+)\s*\(", header))
    assert declared == set(sird.EXPORTS)
    for name in declared:
        assert hasattr(L, name), name


def _create(L, **over):
    from paper_2204_12346_gb300 import sird

    y = over.pop("y", np.arange(31, dtype=float))
    pkw = dict(N=38e6, K=1, spd=10)
    ckw = dict(particles=64, iters=5, lb=[0, 0, 0, 0], ub=[2, 1, 0.1, 1e6])
    for k in list(over):
        if k in ("N", "K", "spd", "cost", "beta_form", "fit_I0", "objective"):
            pkw[k] = over.pop(k)
    ckw.update(over)
    pb, k1 = sird.make_problem(y, **pkw)
    cfg, k2 = sird.make_config(**ckw)
    h = C.c_void_p()
    st = L.sird_pso_create(C.byref(pb), C.byref(cfg), None, C.byref(h))
    return st, L.sird_last_error(None).decode(), h


@pytest.mark.parametrize("over,status", [
    (dict(y=np.array([0.0])), 1),
    (dict(y=np.array([0.0, np.nan, 3.0])), 1),
    (dict(N=-1.0), 1),
    (dict(spd=0), 1),
    (dict(K=0), 1),
    (dict(K=40, lb=[0] * 43, ub=[1] * 43), 1),
    (dict(cost=9), 1),
    (dict(objective=1), 1),  # F_IRD without the I and R series
    (dict(objective=5), 1),
    (dict(particles=0), 1),
    (dict(precision=16), 1),
    (dict(block_size=48), 1),
    (dict(reeval_topk=65), 1),
    (dict(lb=[0, 0, 0, 2e6]), 1),
    (dict(log_scale=[1, 1, 1, 1]), 1),
    (dict(lb=[0, 0, 0, np.inf]), 1),
    (dict(y=np.arange(4097, dtype=float)), 1),  # more than SIRD_MAX_OBS observations
    (dict(N=np.inf), 1),
    (dict(spd=1001), 1),
    (dict(beta_form=2), 1),
    (dict(fit_I0=2), 1),
    (dict(lb=[0, 0, 0, 10.0], ub=[2, 1, 0.1, 5.0]), 1),  # lb > ub
    (dict(launch_mode=9), 1),
    (dict(precision=64, launch_mode=2), 7),  # the persistent and cluster launches are FP32 only
    (dict(precision=64, launch_mode=5), 7),
    (dict(launch_mode=4), 1),  # a batch form is not a handle's launch mode
    (dict(precision=64, block_size=512), 1),
    (dict(particles=(1 << 26) + 1), 1),
    (dict(iters=-1), 1),
])
def test_create_rejects_bad_arguments_without_a_gpu(L, over, status):
    st, msg, h = _create(L, **over)
    assert st == status and msg and not h.value


def _batch_create(L, windows, **over):
    from paper_2204_12346_gb300 import sird

    kw = dict(K=1, spd=10, cost=0, beta_form=0, fit_I0=True, iters=5, lb=[0, 0, 0, 0], ub=[2, 1, 0.1, 1e6],
              log_scale=None, w=0.5, c1=0.5, c2=0.5, particles=64, seed=0, block_size=0)
    kw.update(over)
    pbs, cfgs, keep = sird._batch_structs(windows, **kw)
    h = C.c_void_p()
    st = L.sird_batch_create(len(windows), pbs, cfgs, None, C.byref(h))
    return st, L.sird_last_error(None).decode(), h


@pytest.mark.parametrize("case", ["too_many_particles", "window_particles", "differing_K", "log_lb_zero", "block"])
def test_batch_create_rejects_bad_arguments_without_a_gpu(L, case):
    y = np.arange(31, dtype=float)
    wins = [{"yD": y, "N": 38e6}, {"yD": y[:21], "N": 38e6}]
    over = {}
    if case == "too_many_particles":  # 65 windows of 2^20 particles: more than SIRD_MAX_PARTICLES in all
        wins = [{"yD": y, "N": 38e6, "particles": 1 << 20} for _ in range(65)]
    elif case == "window_particles":
        wins[1]["particles"] = (1 << 20) + 1
    elif case == "differing_K":  # every window must share the model settings
        from paper_2204_12346_gb300 import sird

        pbs, cfgs, keep = sird._batch_structs(wins, K=1, spd=10, cost=0, beta_form=0, fit_I0=True, iters=5,
                                              lb=[0] * 4, ub=[1] * 4, log_scale=None, w=0.5, c1=0.5, c2=0.5,
                                              particles=64, seed=0, block_size=0)
        pbs[1].K = 2
        h = C.c_void_p()
        assert L.sird_batch_create(2, pbs, cfgs, None, C.byref(h)) == 1 and not h.value
        assert "differ" in L.sird_last_error(None).decode()
        return
    elif case == "log_lb_zero":
        over = dict(log_scale=[1, 1, 1, 1])
    elif case == "block":
        over = dict(block_size=48)
    st, msg, h = _batch_create(L, wins, **over)
    assert st == 1 and msg and not h.value, (st, msg)


@pytest.mark.parametrize("case", ["k0", "horizon0", "horizon_big", "null_out", "precision", "bad_problem"])
def test_forecast_rejects_bad_arguments_without_a_gpu(L, case):
    from paper_2204_12346_gb300 import sird

    y = np.arange(31, dtype=float)
    pb, keep = sird.make_problem(y if case != "bad_problem" else y[:1], 38e6)
    th = np.array([[0.2, 0.1, 0.002, 1e4]])
    out = np.zeros(14)
    k, horizon, prec = 1, 14, 64
    k = 0 if case == "k0" else k
    horizon = {"horizon0": 0, "horizon_big": 100001}.get(case, horizon)
    prec = 16 if case == "precision" else prec
    dout = None if case == "null_out" else out.ctypes.data_as(C.POINTER(C.c_double))
    st = L.sird_forecast(C.byref(pb), th.ctypes.data_as(C.POINTER(C.c_double)), k, horizon, dout, prec, None)
    assert st == 1 and L.sird_last_error(None).decode()


@pytest.mark.parametrize("case", ["k_big", "fraction0", "fraction_above_1", "nan_theta", "bands17"])
def test_ensemble_bands_reject_bad_arguments_without_a_gpu(L, case):
    from paper_2204_12346_gb300 import sird

    pb, keep = sird.make_problem(np.arange(31, dtype=float), 38e6)
    k = 4097 if case == "k_big" else 2
    th = np.tile([0.2, 0.1, 0.002, 1e4], (k, 1))
    if case == "nan_theta":
        th[1, 0] = np.nan
    fr = {"fraction0": [0.0], "fraction_above_1": [1.5], "bands17": [0.5] * 17}.get(case, [0.9])
    fr = np.array(fr)
    out = np.zeros(6 * 40 * (1 + 2 * len(fr)))
    dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    st = L.sird_ensemble_bands(C.byref(pb), dp(th), k, 9, dp(fr), len(fr), dp(out), None)
    assert st == 1 and L.sird_last_error(None).decode()


def test_binding_refuses_short_arrays_before_calling_the_library(L):
    # the library reads P bounds, n_obs values of each series and P entries of each theta row:
    # shorter arrays are refused by the binding (no GPU needed to see it)
    from paper_2204_12346_gb300 import sird

    y = np.arange(31, dtype=float)
    assert sird.n_params(4) == 7 and sird.n_params(beta_form=sird.BETA_RAMP, fit_I0=False) == 6
    with pytest.raises(ValueError, match="lb"):
        sird.Calibrator(y, 38e6, K=4, lb=[0] * 6, ub=[1] * 7)
    with pytest.raises(ValueError, match="log_scale"):
        sird.Calibrator(y, 38e6, K=4, lb=[1e-3] * 7, ub=[1] * 7, log_scale=[1] * 3)
    with pytest.raises(ValueError, match="lb and ub"):
        sird.Calibrator(y, 38e6)
    with pytest.raises(ValueError, match="yR"):
        sird.make_problem(y, 38e6, yI=y, yR=y[:10], objective=sird.FIT_IRD)
    with pytest.raises(ValueError, match="lb"):
        sird.Batch([{"yD": y, "N": 38e6}], K=2, lb=[0] * 4, ub=[1] * 5)
    with pytest.raises(ValueError, match="theta"):
        sird.forecast(y, 38e6, np.zeros((3, 5)), 7, K=1)
    with pytest.raises(ValueError, match="theta"):
        sird.ensemble_bands(y, 38e6, np.zeros((3, 3)), 7, K=1)


def test_null_handle_calls_are_safe(L):
    assert L.sird_pso_init(None) == 1
    assert L.sird_pso_step(None, 1) == 1
    assert L.sird_pso_num_params(None) == 0
    f, i = C.c_float(), C.c_int()
    z = (C.c_float * 4)()
    d = (C.c_double * 4)()
    assert L.sird_pso_set_shard(None, 0, 10) == 1
    assert L.sird_pso_shard_best(None, C.byref(f), C.byref(i), z) == 1
    assert L.sird_pso_set_gbest(None, z, 0.0, 0) == 1
    assert L.sird_pso_topk_indexed(None, 1, d, d, C.byref(i)) == 1
    L.sird_pso_destroy(None)


def test_header_is_plain_c_and_a_c_program_calls_the_library(L, tmp_path):
    # the boundary is a C ABI: the header compiles as pedantic C99, and a C program links
    # against the library and gets its argument errors without touching a GPU
    import shutil
    import subprocess

    from paper_2204_12346_gb300 import build

    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use.c"
    src.write_text(
        '#include <stdio.h>\n#include "sird_pso.h"\n'
        "int main(void) {\n"
        "    sird_pso_t h = 0;\n"
        "    sird_status s = sird_pso_create(0, 0, 0, &h);\n"
        '    printf("%d %d %s\\n", (int)s, h == 0, sird_last_error(0));\n'
        "    return s == SIRD_ERR_ARG && h == 0 ? 0 : 1;\n"
        "}\n")
    exe = tmp_path / "use"
    lib_dir = os.path.dirname(build.LIB)
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I",
                        os.path.join(ROOT, "include"), str(src), "-L", lib_dir, "-l:" + os.path.basename(build.LIB),
                        "-Wl,-rpath," + lib_dir, "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert run.returncode == 0, (run.stdout, run.stderr)
    assert run.stdout.split()[0] == "1" and "NULL" in run.stdout


def test_binding_constants_match_the_header():
    # every enumerator and limit the header defines has the same value in the Python binding
    from paper_2204_12346_gb300 import sird

    header = open(os.path.join(ROOT, "include", "sird_pso.h")).read()
    header = re.sub(r"/\*.*?\*/", "", header, flags=re.S)
    values = {m.group(1): int(m.group(2)) for m in re.finditer(r"\bSIRD_([A-Z0-9_]+)\s*=\s*(\d+)", header)}
    assert len(values) >= 20
    for name, v in values.items():
        assert getattr(sird, name) == v, name
    assert re.search(r"#define SIRD_MAX_PARAMS (\d+)", header).group(1) == str(sird.MAX_PARAMS)
