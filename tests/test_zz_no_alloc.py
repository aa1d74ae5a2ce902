"""The allocation-free decode entry point (ldpc_bp_decode_noalloc).

Some callers cannot call cudaMalloc (a real-time receiver that allocates
everything at start-up, a host thread that must never block on the device);
this entry point serves them from a fixed scratch array in the library. These
tests call it through the C ABI and check that two calls in a row give exactly
what ldpc_bp_decode gives on the same inputs (min-sum is bit-exact), and that
a batch too large for the fixed array is refused before any work.

The file is collected last, so a run that stops at the first failure has
already run every other test; it also passes alone in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

from tests import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lx():
    import paper_2203_11854_gb300 as lx
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    lx.load_library()
    return lx


def decode_noalloc_abi(lx, code, llr, opts):
    """Call ldpc_bp_decode_noalloc through the C ABI with caller-owned outputs."""
    B = llr.shape[0]
    llr_out = torch.empty((B, code.n), dtype=torch.float32, device="cuda")
    bits = torch.empty((B, (code.k + 31) // 32), dtype=torch.int32, device="cuda")
    its = torch.empty((B,), dtype=torch.int32, device="cuda")
    st = lx.load_library().ldpc_bp_decode_noalloc(code.handle, llr.data_ptr(), B, C.byref(opts), llr_out.data_ptr(),
                                                  bits.data_ptr(), its.data_ptr(),
                                                  torch.cuda.current_stream().cuda_stream)
    assert st == 0, lx.ldpcx_status_str(st)
    return llr_out, bits, its


@pytest.mark.parametrize("bg,Z,punct,B,algo,prec,early", [
    (1, 384, 2, 40, 0, 1, False),   # BG1-shaped Z=384, FP16 min-sum (the headline decoder)
    (1, 384, 2, 24, 0, 0, True),    # FP32 messages, early stop
    (2, 64, 0, 150, 0, 2, False),   # BG2-shaped Z=64, 6-bit messages, several CTAs + ragged tail
    (2, 8, 0, 100, 2, 0, True),     # flooding min-sum
])
def test_noalloc_matches_ldpc_bp_decode_twice(lx, bg, Z, punct, B, algo, prec, early):
    code = lx.qc_ldpc_build(bg, Z, punct_cols=punct)
    opts = lx.DecodeOpts(algo, 12, prec, int(early), 0.5, 20.0, None)
    for call, seed in enumerate((101, 202)):  # two calls in a row, different inputs
        llr = torch.from_numpy(inputs.gaussian_llrs(np.zeros((B, code.n_tx), np.uint8), 1.5, seed)).cuda()
        got = decode_noalloc_abi(lx, code, llr, opts)
        ref = lx.ldpc_bp_decode(code, llr, algo=algo, iters=12, msg_prec=prec, early_stop=early, llr_out=True)
        torch.cuda.synchronize()
        for g, r in zip(got, ref):
            assert torch.equal(g, r), f"call {call}"
    assert lx.ldpcx_sync_status()[0] == 0


def test_noalloc_refuses_batches_beyond_the_array(lx):
    code = lx.qc_ldpc_build(1, 384, punct_cols=2)
    opts = lx.DecodeOpts(0, 20, 1, 0, 0.5, 20.0, None)  # FP16 messages: at most 138 codewords
    llr = torch.zeros((139, code.n_tx), dtype=torch.float32, device="cuda")
    st = lx.load_library().ldpc_bp_decode_noalloc(code.handle, llr.data_ptr(), 139, C.byref(opts), None, None,
                                                  None, None)
    assert st == -4  # LDPCX_E_WORKSPACE
    ok = lx.load_library().ldpc_bp_decode_noalloc(code.handle, llr.data_ptr(), 138, C.byref(opts), None, None,
                                                  None, None)
    assert ok == 0
    torch.cuda.synchronize()
