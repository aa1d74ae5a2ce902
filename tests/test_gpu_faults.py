"""Failure detection on the GPU path without a GPU fault: an injected host
allocation failure (ldpcx_fault_set) at the first device use of a code -- the
upload of its tables -- makes every entry point that uploads them return
LDPCX_E_NOMEM before any kernel runs, with the caller's outputs untouched;
the call after it succeeds. The allocation-free decode performs no allocation
at all, so an armed fault survives it."""
import ctypes as C

import numpy as np
import pytest

from tests import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
E_NOMEM = -3


@pytest.fixture(scope="module")
def lx():
    import paper_2203_11854_gb300 as lx
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    lx.load_library()
    yield lx
    lx.ldpcx_fault_set(lx.FAULT_NONE)


def fresh(lx):
    return lx.qc_ldpc_build(2, 16, punct_cols=2)  # no device tables yet


def expect_nomem(lx, fn, *outs):
    before = [o.clone() for o in outs]
    lx.ldpcx_fault_set(lx.FAULT_ALLOC, 0)
    with pytest.raises(lx.LdpcxError) as e:
        fn()
    assert e.value.status == E_NOMEM
    torch.cuda.synchronize()
    for o, b in zip(outs, before):
        assert torch.equal(o, b)  # untouched
    fn()  # one shot: the retry runs
    torch.cuda.synchronize()


def sentinel(shape, dtype):
    return torch.full(shape, 77, dtype=dtype, device="cuda")


def test_decode_first_use(lx):
    code = fresh(lx)
    B = 9
    llr = torch.from_numpy(inputs.gaussian_llrs(np.zeros((B, code.n_tx), np.uint8), 2.0, 3)).cuda()
    llr_out = sentinel((B, code.n), torch.float32)
    bits = sentinel((B, (code.k + 31) // 32), torch.int32)
    its = sentinel((B,), torch.int32)
    expect_nomem(lx, lambda: lx.ldpc_bp_decode(code, llr, iters=5, llr_out=llr_out, bits_out=bits, iters_out=its),
                 llr_out, bits, its)


def test_transmitter_first_use(lx):
    code = fresh(lx)
    B = 5
    no = torch.full((1,), 0.5, device="cuda")
    y = sentinel((B, code.n_tx // 2, 2), torch.float32)
    info = sentinel((B, (code.k + 31) // 32), torch.int32)
    expect_nomem(lx, lambda: lx.sim_tx(code, 1, 0, B, 4, no, y_out=y, info_out=info), y, info)
    code2 = fresh(lx)
    cw = sentinel((B, (code2.n + 31) // 32), torch.int32)
    expect_nomem(lx, lambda: lx.sim_codewords(code2, 1, 0, B, out=cw), cw)


def test_mixed_first_use(lx):
    code = fresh(lx)
    llr = torch.from_numpy(inputs.gaussian_llrs(np.zeros((6, code.n_tx), np.uint8), 2.0, 4)).cuda()
    expect_nomem(lx, lambda: lx.ldpc_bp_decode_mixed([(code, llr)], iters=4))


def test_sim_run_first_use(lx):
    code = fresh(lx)
    import paper_2203_11854_gb300 as m
    cfg, keep = m._sim_config(code, [2.0], **{**m._SIM_DEFAULTS, "batch": 64})
    ws = torch.empty(lx.sim_workspace(code, [2.0], batch=64), dtype=torch.uint8, device="cuda")
    out = (lx.SimCounts * 1)()
    out[0].bits = 12345
    n = C.c_int(-7)
    L = lx.load_library()
    lx.ldpcx_fault_set(lx.FAULT_ALLOC, 0)
    st = L.sim_run(C.byref(cfg), out, C.byref(n), ws.data_ptr(), ws.numel(), None)
    assert st == E_NOMEM and out[0].bits == 12345 and n.value == -7
    assert L.sim_run(C.byref(cfg), out, C.byref(n), ws.data_ptr(), ws.numel(), None) == 0
    assert n.value == 1 and out[0].bits == 64 * code.k


def test_polar_first_use(lx):
    pc = lx.polar_build(7, 64, 1.0)
    B = 4
    no = torch.full((1,), 0.5, device="cuda")
    y = sentinel((B, pc.N), torch.float32)
    d = sentinel((B, (pc.k_data + 31) // 32), torch.int32)
    expect_nomem(lx, lambda: lx.polar_sim_tx(pc, 1, 0, B, no, y_out=y, data_out=d), y, d)


def test_noalloc_performs_no_allocation(lx):
    code = fresh(lx)
    B = 6
    llr = torch.from_numpy(inputs.gaussian_llrs(np.zeros((B, code.n_tx), np.uint8), 2.0, 5)).cuda()
    lx.ldpcx_fault_set(lx.FAULT_ALLOC, 0)
    try:
        got = lx.ldpc_bp_decode_noalloc(code, llr, iters=5, msg_prec=lx.MSG_F16)
        torch.cuda.synchronize()
        # the fault is still armed: the next allocation (this code's first table upload) fails
        with pytest.raises(lx.LdpcxError) as e:
            lx.ldpc_bp_decode(code, llr, iters=5, msg_prec=lx.MSG_F16)
        assert e.value.status == E_NOMEM
    finally:
        lx.ldpcx_fault_set(lx.FAULT_NONE)
    ref = lx.ldpc_bp_decode(code, llr, iters=5, msg_prec=lx.MSG_F16)
    assert torch.equal(got[1], ref[1]) and torch.equal(got[2], ref[2])
