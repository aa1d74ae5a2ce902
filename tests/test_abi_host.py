"""CPU checks of the C ABI: the library builds, loads and exports every symbol
that include/ldpcx.h declares; host-side code construction matches the oracle;
argument validation answers before any device work."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ldpcx.h")


@pytest.fixture(scope="module")
def lx():
    import paper_2203_11854_gb300 as lx
    lx._build.build()
    lx.load_library()
    return lx


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^[A-Za-z_][\w\s\*]*?\b(\w+)\s*\(", text, flags=re.M)) - {"if", "while"})


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["qc_ldpc_build", "demap_app", "ldpc_bp_decode", "sim_run", "sim_tx", "sim_count",
                     "ldpc_bp_workspace", "qc_ldpc_free", "qc_ldpc_info", "ldpcx_sync_status"]:
        assert required in names


def test_every_declared_symbol_is_exported(lx):
    L = C.CDLL(lx.library_path())
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing


def test_no_oracle_in_product():
    pkg = os.path.join(ROOT, "paper_2203_11854_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src and "ldpc_oracle" not in src, f


@pytest.mark.parametrize("bg,Z,rows_kept", [(1, 384, 0), (2, 8, 0), (2, 64, 0), (1, 16, 13), (2, 128, 7)])
def test_code_construction_matches_oracle(lx, orc, bg, Z, rows_kept):
    code = lx.qc_ldpc_build(bg, Z, rows_kept=rows_kept, punct_cols=2 if bg == 1 else 0)
    S_ref, kb = orc.base_matrix(bg, Z, 1 if bg == 1 else 2, rows_kept)
    assert (code.base() == S_ref).all()
    assert code.kb == kb and code.rows == S_ref.shape[0] and code.cols == S_ref.shape[1]
    assert code.nnz == int((S_ref >= 0).sum())
    assert code.edges == code.nnz * Z
    assert code.n == S_ref.shape[1] * Z and code.k == kb * Z
    assert code.max_row_deg == int((S_ref >= 0).sum(axis=1).max())
    if bg == 1:
        assert code.p0 == 2 * Z and code.n_tx == code.n - 2 * Z


def test_golden_base_matrices(lx):
    import json
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "base_matrices.json")))
    for entry in gold["codes"]:
        code = lx.qc_ldpc_build(entry["bg"], entry["Z"], seed=entry["seed"])
        assert code.base().tolist() == entry["S"], entry["name"]


def test_argument_validation(lx):
    L = lx.load_library()
    h = C.c_void_p()
    for bad in [lx.CodeParams(3, 8, 1, 0, 0, 0), lx.CodeParams(1, 1, 1, 0, 0, 0), lx.CodeParams(1, 385, 1, 0, 0, 0),
                lx.CodeParams(1, 8, 1, 3, 0, 0), lx.CodeParams(1, 8, 1, 47, 0, 0), lx.CodeParams(2, 8, 1, 0, 11, 0),
                lx.CodeParams(2, 8, 1, 0, 0, 10000)]:
        assert L.qc_ldpc_build(C.byref(bad), C.byref(h)) == -1
    assert L.qc_ldpc_build(None, C.byref(h)) == -1
    code = lx.qc_ldpc_build(2, 8)
    o = lx.DecodeOpts(0, 20, 0, 0, 0.5, 20.0, None)
    ws = C.c_size_t(0)
    assert L.ldpc_bp_workspace(code.handle, 10, C.byref(o), C.byref(ws)) == 0
    assert ws.value == 10 * ((197 * 8 + 127) // 128 * 128) * 4
    for fld, val in [("algo", 4), ("iters", 0), ("iters", 1001), ("msg_prec", 3), ("early_stop", 2),
                     ("offset", -1.0), ("clamp", 0.0)]:
        o2 = lx.DecodeOpts(0, 20, 0, 0, 0.5, 20.0, None)
        setattr(o2, fld, val)
        assert L.ldpc_bp_workspace(code.handle, 10, C.byref(o2), C.byref(ws)) == -1, fld
    spa_fix6 = lx.DecodeOpts(1, 20, 2, 0, 0.5, 20.0, None)
    assert L.ldpc_bp_workspace(code.handle, 10, C.byref(spa_fix6), C.byref(ws)) == -2
    weighted_layered = lx.DecodeOpts(0, 20, 0, 0, 0.5, 20.0, 1234)
    assert L.ldpc_bp_workspace(code.handle, 10, C.byref(weighted_layered), C.byref(ws)) == -1
    # decode: null input, too-small workspace; B = 0 is a no-op
    assert L.ldpc_bp_decode(code.handle, None, 4, C.byref(o), None, None, None, None, 0, None) == -1
    assert L.ldpc_bp_decode(code.handle, 4096, 4, C.byref(o), None, None, None, 256, 16, None) == -4
    assert L.ldpc_bp_decode(code.handle, None, 0, C.byref(o), None, None, None, None, 0, None) == 0
    # demapper and transmitter enums
    assert L.demap_app(16, 16, 0, 1, 1, 3, 0, 20.0, 16, None) == -1
    assert L.demap_app(16, 16, 2, 1, 1, 2, 0, 20.0, 16, None) == -1
    assert L.demap_app(16, 16, 0, 1, 1, 2, 5, 20.0, 16, None) == -1
    assert L.sim_tx(code.handle, 1, 0, 4, 3, 16, 0, 16, 16, None) == -1
    assert L.sim_count(16, 16, None, 4, 0, 16, None) == -1
    # rate matching: buffer, start, length and rows checked before any launch; B = 0 is a no-op
    nb = code.n - code.p0
    for k0, ncb, E, qm in [(0, 0, 8, 1), (3, 3, 8, 1), (-1, 8, 8, 1), (0, nb + 1, 8, 1), (0, 8, 0, 1), (0, 8, 9, 2),
                           (0, 8, 9, 3)]:
        assert L.rate_match(code.handle, 16, 4, k0, ncb, E, qm, 16, None) == -1, (k0, ncb, E, qm)
        assert L.rate_recover(code.handle, 16, 4, k0, ncb, E, qm, 16, None) == -1, (k0, ncb, E, qm)
    assert L.rate_match(code.handle, None, 4, 0, nb, 8, 1, 16, None) == -1
    assert L.rate_match(code.handle, None, 0, 0, nb, 8, 1, None, None) == 0
    # user base matrices: the transmitter refuses an unencodable code before any launch
    S = code.base().copy()
    S[5, 10 + 7] = 1  # extension row 5 reads a later parity column
    ucode = lx.qc_ldpc_build_base(S, 8, 10)
    assert ucode.encodable == 0
    assert L.sim_tx(ucode.handle, 1, 0, 4, 2, 16, 0, 16, 16, None) == -2
    assert L.sim_codewords(ucode.handle, 1, 0, 4, 16, None) == -2
    assert lx.ldpcx_status_str(-4).startswith("LDPCX_E_WORKSPACE")
    # phi: the form is one of the three, checked before any launch
    for fast in (-1, 3):
        assert L.ldpcx_phi(16, 16, 4, fast, None) == -1, fast
    assert L.ldpcx_phi(None, None, 0, 2, None) == 0


@pytest.mark.skipif(os.environ.get("CUDA_VISIBLE_DEVICES") is None and __import__("torch").cuda.is_available(),
                    reason="checks the no-device path")
def test_no_device_is_reported(lx):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    L = lx.load_library()
    code = lx.qc_ldpc_build(2, 8)
    o = lx.DecodeOpts(0, 20, 0, 0, 0.5, 20.0, None)
    st = L.ldpc_bp_decode(code.handle, 4096, 4, C.byref(o), None, None, None, 4096 * 256, 1 << 30, None)
    assert st in (-8, -5)
    assert L.ldpcx_sync_status(None, None) == -8


def test_shorten_host_checks(lx):
    """qc_ldpc_shorten is host work: sizes of the derived code and its argument checks, no GPU needed."""
    mother = lx.qc_ldpc_build(2, 52, punct_cols=2)
    sc = lx.qc_ldpc_shorten(mother, 500)
    assert (sc.k, sc.n_fill, sc.n_tx, sc.n, sc.p0) == (500, 20, 2580, 2704, 104)
    assert (sc.nnz, sc.rows, sc.cols, sc.kb) == (mother.nnz, mother.rows, mother.cols, mother.kb)
    assert (sc.base() == mother.base()).all()
    assert lx.qc_ldpc_shorten(mother, 520).n_fill == 0
    h = C.c_void_p()
    L = lx.load_library()
    for k in (103, 521, -1):  # below the punctured columns, above kb Z
        assert L.qc_ldpc_shorten(mother.handle, k, C.byref(h)) == -1
    assert L.qc_ldpc_shorten(sc.handle, 400, C.byref(h)) == -1  # a shortened code is not shortened again
    assert L.qc_ldpc_shorten(None, 400, C.byref(h)) == -1
    # fillers outside the transmitted span
    trunc = lx.qc_ldpc_build(2, 52, punct_cols=2, n_tx=300)
    assert L.qc_ldpc_shorten(trunc.handle, 500, C.byref(h)) == -1
    del mother  # the derived code keeps its own copy of the tables
    assert lx.qc_ldpc_info(sc).k == 500


def test_qam_map_awgn_argument_checks(lx):
    L = lx.load_library()
    one = C.c_void_p(16)  # never dereferenced: every call below returns before device work
    assert L.qam_map_awgn(one, 0, 8, 4, 1, 0, one, 0, one, None) == 0     # B = 0: nothing to do
    assert L.qam_map_awgn(one, 2, 10, 4, 1, 0, one, 0, one, None) == -1   # m does not divide E
    assert L.qam_map_awgn(one, 2, 8, 3, 1, 0, one, 0, one, None) == -1    # m not a constellation size
    assert L.qam_map_awgn(one, 2, 8, 4, 1, 0, one, 2, one, None) == -1    # N0 stride 0 or 1
    assert L.qam_map_awgn(None, 2, 8, 4, 1, 0, one, 0, one, None) == -1   # null bits


def test_decode_qam_argument_checks(lx):
    """ldpc_bp_decode_qam refuses bad arguments and the flooding schedules before any device work."""
    L = lx.load_library()
    code = lx.qc_ldpc_build(2, 8)  # n_tx = 416: m = 1, 2, 4, 8 divide it, m = 6 does not
    one = C.c_void_p(16)  # never dereferenced: every call below returns before device work

    def call(B=2, m=4, stride=0, method=lx.DEMAP_MAXLOG, dclamp=20.0, algo=lx.LAYERED_MINSUM, y=one, ws=None, nws=0):
        o = lx.DecodeOpts(algo, 20, lx.MSG_F16, 0, 0.5, 20.0, None)
        return L.ldpc_bp_decode_qam(code.handle, y, one, stride, B, m, method, dclamp, C.byref(o), None, one, None,
                                    ws, nws, None)

    assert call(B=0) == 0                               # nothing to do
    assert call(m=3) == -1                              # not a constellation size
    assert call(m=6) == -1                              # m does not divide n_tx
    assert call(stride=2) == -1                         # N0 stride 0 or 1
    assert call(method=2) == -1                         # demapper method
    assert call(dclamp=0.0) == -1                       # demapper clamp > 0
    assert call(dclamp=float("inf")) == -1              # and finite
    assert call(algo=lx.FLOOD_SPA) == -2                # flooding reads the channel LLRs every iteration
    assert call(algo=lx.FLOOD_MINSUM) == -2
    assert call(y=None) == -1                           # null symbols
    assert call() == -4                                 # missing workspace
    assert L.ldpc_bp_decode_qam(None, one, one, 0, 2, 4, 0, 20.0, None, None, one, None, None, 0, None) == -1


def test_ckpt_bytes_hold_messages_and_app(lx):
    """The differentiable decode's checkpoints: per iteration but the last, every codeword's messages (edges
    rounded up to 128 floats) and its APP values (n rounded up to 32 floats)."""
    code = lx.qc_ldpc_build(2, 8)  # 197 blocks x 8 = 1576 edges, n = 416
    per_cw = (1576 + 127) // 128 * 128 + (416 + 31) // 32 * 32
    assert lx.ldpc_bp_ckpt_bytes(code, 10, iters=8) == 4 * 7 * 10 * per_cw
    assert lx.ldpc_bp_ckpt_bytes(code, 3, iters=1) == 4 * 1 * 3 * per_cw  # one slot even without a stored iteration
