"""The allocation-free decode entry point (ldpc_bp_decode_noalloc).

Some callers cannot call cudaMalloc (a real-time receiver that allocates
everything at start-up, a host thread that must never block on the device);
this entry point serves them from a fixed scratch array in the library. These
tests call it through the C ABI and check that two calls in a row give exactly
what ldpc_bp_decode gives on the same inputs (it runs the same kernel), for
min-sum (check-node state) and sum-product (per-edge messages, layered and
weighted flooding); that its min-sum output equals the oracle's FP32 replay;
and that a batch too large for the fixed array is refused before any work.

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


@pytest.mark.parametrize("bg,Z,punct,B,algo,prec,early,weighted", [
    (1, 384, 2, 40, 0, 1, False, False),   # BG1-shaped Z=384, FP16 min-sum (the headline decoder)
    (1, 384, 2, 24, 0, 0, True, False),    # FP32 messages, early stop
    (1, 384, 2, 153, 0, 1, False, False),  # FP16 min-sum at the array's limit (218112-byte state)
    (2, 64, 0, 150, 0, 2, False, False),   # BG2-shaped Z=64, 6-bit messages, several CTAs + ragged tail
    (1, 128, 2, 9, 0, 1, True, False),     # BG1-shaped Z=128, FP16 min-sum, early stop
    (2, 8, 0, 100, 2, 0, True, False),     # flooding min-sum
    (1, 384, 2, 12, 1, 0, False, False),   # layered sum-product, FP32 messages (compiled schedule)
    (1, 384, 2, 12, 1, 1, False, False),   # layered sum-product, FP16 messages
    (2, 64, 0, 33, 3, 0, False, True),     # weighted flooding sum-product, FP32
    (2, 64, 0, 33, 3, 1, True, False),     # flooding sum-product, FP16, early stop
])
def test_noalloc_matches_ldpc_bp_decode_twice(lx, bg, Z, punct, B, algo, prec, early, weighted):
    code = lx.qc_ldpc_build(bg, Z, punct_cols=punct)
    iters = 12
    w = None
    if weighted:
        w = torch.from_numpy((0.6 + 0.8 * inputs.rng(5).random((iters, code.nnz))).astype(np.float32)).cuda()
    opts = lx.DecodeOpts(algo, iters, prec, int(early), 0.5, 20.0, None if w is None else w.data_ptr())
    for call, seed in enumerate((101, 202)):  # two calls in a row, different inputs
        llr = torch.from_numpy(inputs.gaussian_llrs(np.zeros((B, code.n_tx), np.uint8), 1.5, seed)).cuda()
        got = decode_noalloc_abi(lx, code, llr, opts)
        ref = lx.ldpc_bp_decode(code, llr, algo=algo, iters=iters, msg_prec=prec, early_stop=early, llr_out=True,
                                weights=w)
        torch.cuda.synchronize()
        for g, r in zip(got, ref):
            assert torch.equal(g, r), f"call {call}"
    assert lx.ldpcx_sync_status()[0] == 0


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_noalloc_minsum_equals_oracle_replay(lx, orc, prec):
    """Layered min-sum through the allocation-free entry point against the oracle's FP32 replay with the
    same message store: output LLRs, hard decisions and iteration counts bit for bit."""
    ocode = orc.Code(2, 64)
    code = lx.qc_ldpc_build(2, 64)
    B = 23
    cw = ocode.encoder.encode(inputs.info_bits(41, B, ocode.k))
    L = inputs.gaussian_llrs(cw, 2.2, 42)
    opts = lx.DecodeOpts(0, 8, prec, 1, 0.5, 20.0, None)
    llr, bits, its = decode_noalloc_abi(lx, code, torch.from_numpy(np.ascontiguousarray(L)).cuda(), opts)
    app, hard, oits = orc.decode(ocode.graph, L.astype(np.float64), algo=0, schedule=0, iters=8, prec=1, store=prec,
                                 early_stop=True)
    assert np.array_equal(llr.cpu().numpy(), app.astype(np.float32))
    w = bits.cpu().numpy().view(np.uint32)
    got = ((w[:, :, None] >> np.arange(32, dtype=np.uint32)) & 1).reshape(B, -1)[:, :ocode.k]
    assert np.array_equal(got, hard[:, :ocode.k])
    assert np.array_equal(its.cpu().numpy(), oits)


@pytest.mark.parametrize("algo,prec,limit", [
    (0, 1, 153),  # layered min-sum, FP16: core-row state + per-edge extension rows, 218112 bytes per codeword
    (0, 0, 118),  # FP32 state: 282624 bytes
    (0, 2, 307),  # 6-bit: core-row state + per-edge extension rows, 109056 bytes
    (1, 1, 138),  # layered sum-product, FP16 per-edge messages: 242688 bytes
])
def test_noalloc_refuses_batches_beyond_the_array(lx, algo, prec, limit):
    code = lx.qc_ldpc_build(1, 384, punct_cols=2)
    # the limit follows from the decoder's own per-codeword bytes and the 256-byte-rounded tables
    _, per_cw = lx.ldpc_bp_msg_format(code, algo=algo, iters=20, msg_prec=prec)
    tables = (4 * (code.nnz + code.rows + 1) + 255) // 256 * 256
    assert limit == ((32 << 20) - tables) // per_cw
    opts = lx.DecodeOpts(algo, 20, prec, 0, 0.5, 20.0, None)
    llr = torch.zeros((limit + 1, code.n_tx), dtype=torch.float32, device="cuda")
    st = lx.load_library().ldpc_bp_decode_noalloc(code.handle, llr.data_ptr(), limit + 1, C.byref(opts), None,
                                                  None, None, None)
    assert st == -4  # LDPCX_E_WORKSPACE
    # an absurd batch is refused without forming an overflowing product
    st = lx.load_library().ldpc_bp_decode_noalloc(code.handle, llr.data_ptr(), 1 << 62, C.byref(opts), None,
                                                  None, None, None)
    assert st == -4
    ok = lx.load_library().ldpc_bp_decode_noalloc(code.handle, llr.data_ptr(), limit, C.byref(opts), None, None,
                                                  None, None)
    assert ok == 0
    torch.cuda.synchronize()
