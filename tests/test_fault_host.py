"""Host-side failure detection without a GPU: the allocation fault injector
(ldpcx_fault_set and the LDPCX_FAULT environment variable) drives every host
allocation of the library into its LDPCX_E_NOMEM path, with the caller's
output handle untouched; a sweep checkpoint that this library did not write
for the same sweep is refused (LDPCX_E_IO) before any device work."""
import ctypes as C
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
E_INVAL, E_NOMEM, E_IO = -1, -3, -9
SENTINEL = 0x5EED


@pytest.fixture(scope="module")
def lx():
    import paper_2203_11854_gb300 as lx
    lx._build.build()
    lx.load_library()
    yield lx
    lx.ldpcx_fault_set(lx.FAULT_NONE)


def builders(lx):
    L = lx.load_library()
    mother = lx.qc_ldpc_build(2, 16, punct_cols=2)
    S = np.ascontiguousarray(mother.base(), dtype=np.int16)
    bp = lx.BaseParams(S.shape[0], S.shape[1], 10, 16, S.ctypes.data, 2, 0)
    cp = lx.CodeParams(2, 16, 2, 0, 2, 0)
    return {
        "qc_ldpc_build": lambda h: L.qc_ldpc_build(C.byref(cp), C.byref(h)),
        "qc_ldpc_build_base": lambda h: L.qc_ldpc_build_base(C.byref(bp), C.byref(h)),
        "qc_ldpc_shorten": lambda h: L.qc_ldpc_shorten(mother.handle, 150, C.byref(h)),
        "polar_build": lambda h: L.polar_build(8, 128, 0.0, 0, 0, C.byref(h)),
    }, (S, mother)


@pytest.mark.parametrize("name", ["qc_ldpc_build", "qc_ldpc_build_base", "qc_ldpc_shorten", "polar_build"])
def test_injected_allocation_failure(lx, name):
    calls, _keep = builders(lx)
    call = calls[name]
    L = lx.load_library()
    free = L.polar_free if name == "polar_build" else L.qc_ldpc_free
    lx.ldpcx_fault_set(lx.FAULT_ALLOC, 0)
    h = C.c_void_p(SENTINEL)
    assert call(h) == E_NOMEM
    assert h.value == SENTINEL  # the output is untouched
    # one shot: the next allocation succeeds
    assert call(h) == 0 and h.value not in (None, SENTINEL)
    free(h)
    # after = 1: one allocation passes, the second fails
    lx.ldpcx_fault_set(lx.FAULT_ALLOC, 1)
    h1, h2 = C.c_void_p(SENTINEL), C.c_void_p(SENTINEL)
    assert call(h1) == 0 and call(h2) == E_NOMEM and h2.value == SENTINEL
    free(h1)
    # disarmed
    lx.ldpcx_fault_set(lx.FAULT_ALLOC, 0)
    lx.ldpcx_fault_set(lx.FAULT_NONE)
    assert call(h) == 0
    free(h)


def test_fault_set_argument_checks(lx):
    L = lx.load_library()
    assert L.ldpcx_fault_set(7, 0) == E_INVAL
    assert L.ldpcx_fault_set(lx.FAULT_ALLOC, -1) == E_INVAL
    assert L.ldpcx_fault_set(lx.FAULT_NONE, 0) == 0


def test_fault_from_environment(lx):
    prog = ("import ctypes as C, paper_2203_11854_gb300 as lx\n"
            "L = lx.load_library()\n"
            "p = lx.CodeParams(2, 8, 2, 0, 0, 0)\n"
            "r = []\n"
            "for _ in range(3):\n"
            "    h = C.c_void_p(7)\n"
            "    r.append(L.qc_ldpc_build(C.byref(p), C.byref(h)))\n"
            "print(r)\n")
    env = dict(os.environ, LDPCX_FAULT="alloc:1", PYTHONPATH=ROOT)
    out = subprocess.run([sys.executable, "-c", prog], env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == f"[0, {E_NOMEM}, 0]"


def sim_cfg(lx, code, path, seed=0x5EED):
    import paper_2203_11854_gb300 as m
    kw = {**m._SIM_DEFAULTS, "ckpt_path": path, "seed": seed}
    return m._sim_config(code, [1.0, 2.0], **kw)


def test_checkpoint_of_another_sweep_is_refused_before_device_work(lx, tmp_path):
    code = lx.qc_ldpc_build(2, 16, punct_cols=2)
    L = lx.load_library()
    path = str(tmp_path / "ck.json")
    fake_ws = C.c_void_p(1 << 20)  # never dereferenced: each call below returns before device work
    out = (lx.SimCounts * 2)()
    n = C.c_int(-1)
    # the library's own layout (one item per line), with a fingerprint of no sweep of this test
    foreign = ('{\n "format": "ldpcx-sim-checkpoint",\n "version": 1,\n "fingerprint": "0123456789abcdef",\n'
               ' "next_point": 0,\n "next_cw": 0,\n "finished": 1,\n "points": [\n ]\n}\n')
    json.loads(foreign)
    cases = {"foreign fingerprint": foreign, "not a checkpoint": json.dumps({"hello": 1}, indent=1)}
    for what, text in cases.items():
        with open(path, "w") as f:
            f.write(text)
        cfg, keep = sim_cfg(lx, code, path)
        assert L.sim_run(C.byref(cfg), out, C.byref(n), fake_ws, 1 << 40, None) == E_IO, what
        assert n.value == -1  # outputs untouched
    with open(path, "w") as f:
        f.write("{\n truncated")
    cfg, keep = sim_cfg(lx, code, path)
    assert L.sim_run(C.byref(cfg), out, C.byref(n), fake_ws, 1 << 40, None) == E_IO
