"""The library's NVTX ranges reach a profiler (CPU only).

A minimal NVTX tool, built here with gcc, stands in for the profiler: NVTX v3 loads the library
named by NVTX_INJECTION64_PATH, calls its InitializeInjectionNvtx2 and routes domain creation,
range push and range pop to it.  The entry points below fail their argument checks before any
CUDA call, so no GPU is needed, yet each opens and closes its range.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INCLUDE = "/usr/local/cuda/include"

TOOL_SRC = r"""
#include <nvtx3/nvToolsExt.h>
#include <stdio.h>
#include <string.h>

static char log_buf[1 << 16];
static size_t log_len = 0;

static void put(const char* kind, nvtxDomainHandle_t d, const char* msg) {
    int n = snprintf(log_buf + log_len, sizeof(log_buf) - log_len, "%s %s %s\n", kind,
                     d ? (const char*)d : "-", msg ? msg : "-");
    if (n > 0 && log_len + (size_t)n < sizeof(log_buf)) log_len += (size_t)n;
}

/* the domain handle is the domain's name, kept for the life of the process */
static char names[16][64];
static int n_names = 0;

static nvtxDomainHandle_t create(const char* name) {
    if (n_names >= 16) return 0;
    strncpy(names[n_names], name, 63);
    return (nvtxDomainHandle_t)names[n_names++];
}

static int push(nvtxDomainHandle_t d, const nvtxEventAttributes_t* a) {
    put("push", d, a && a->messageType == NVTX_MESSAGE_TYPE_ASCII ? a->message.ascii : 0);
    return 0;
}

static int pop(nvtxDomainHandle_t d) {
    put("pop", d, 0);
    return 0;
}

int InitializeInjectionNvtx2(NvtxGetExportTableFunc_t get) {
    const NvtxExportTableCallbacks* cb = (const NvtxExportTableCallbacks*)get(NVTX_ETID_CALLBACKS);
    NvtxFunctionTable t = 0;
    unsigned int n = 0;
    if (!cb || !cb->GetModuleFunctionTable(NVTX_CB_MODULE_CORE2, &t, &n) || n < NVTX_CBID_CORE2_DomainCreateA)
        return 0;
    *t[NVTX_CBID_CORE2_DomainCreateA] = (NvtxFunctionPointer)create;
    *t[NVTX_CBID_CORE2_DomainRangePushEx] = (NvtxFunctionPointer)push;
    *t[NVTX_CBID_CORE2_DomainRangePop] = (NvtxFunctionPointer)pop;
    return 1;
}

/* the recorded events, one per line */
const char* tool_log(void) { return log_buf; }
"""

CALLER = r"""
import ctypes as C, os, sys
sys.path.insert(0, sys.argv[1])
from paper_2204_12346_gb300 import sird
L = sird.lib()
h = C.c_void_p()
assert L.sird_batch_create(0, None, None, None, C.byref(h)) == sird.ERR_ARG
assert L.sird_forecast(None, None, 0, 0, None, 64, None) == sird.ERR_ARG
tool = C.CDLL(os.environ["NVTX_INJECTION64_PATH"])
tool.tool_log.restype = C.c_char_p
sys.stdout.write(tool.tool_log().decode())
"""


def test_entry_points_open_and_close_their_ranges(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None or not os.path.exists(os.path.join(CUDA_INCLUDE, "nvtx3", "nvToolsExt.h")):
        pytest.skip("no C compiler or NVTX headers")
    from paper_2204_12346_gb300 import build

    build.build()
    (tmp_path / "tool.c").write_text(TOOL_SRC)
    tool = tmp_path / "libtool.so"
    r = subprocess.run([gcc, "-std=c11", "-shared", "-fPIC", "-I", CUDA_INCLUDE, str(tmp_path / "tool.c"), "-o",
                        str(tool), "-ldl"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    (tmp_path / "caller.py").write_text(CALLER)
    env = dict(os.environ, NVTX_INJECTION64_PATH=str(tool))
    run = subprocess.run([sys.executable, str(tmp_path / "caller.py"), ROOT], env=env, capture_output=True, text=True,
                         timeout=300)
    assert run.returncode == 0, run.stderr
    events = [tuple(l.split()) for l in run.stdout.splitlines()]
    assert events == [("push", "sird_pso", "sird_batch_create"), ("pop", "sird_pso", "-"),
                      ("push", "sird_pso", "sird_forecast"), ("pop", "sird_pso", "-")], events
