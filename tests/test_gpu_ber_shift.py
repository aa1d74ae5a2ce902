"""BER-curve shift at BER 1e-4 of the GPU decoders against the FP64 oracle.

Workloads: BG1-shaped Z=384 (2Z punctured), 16-QAM and 256-QAM, max-log
demapper, layered offset min-sum (0.5), 20 iterations. A coarse GPU FP32 sweep finds the two
Eb/N0 points that bracket BER 1e-4; at those points the FP64 oracle, and the
GPU decoder with FP32, FP16 and 6-bit messages, decode the same codewords with
the same noise draws (Philox seed and codeword range). The Eb/N0 at 1e-4 is
interpolated in log10(BER) on a 0.1 dB grid; FP32 and FP16 messages must stay
within 0.05 dB of the FP64 oracle (the 6-bit result is reported).
"""
import os

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SEED = 0x1DBC | (2 << 32)
N = 12288  # codewords per point for the paired comparison


@pytest.mark.parametrize("m,start", [(4, 2.5), (8, 7.0)])
def test_ber_shift_at_1e4(orc, m, start):
    import paper_2203_11854_gb300 as lx
    from paper_2203_11854_gb300 import ber
    assert torch.cuda.is_available()
    lx.load_library()
    code = lx.qc_ldpc_build(1, 384, punct_cols=2)
    grid = [start + 0.25 * i for i in range(17)]
    br, pts = ber.bracket(code, grid, codewords=16384, seed=SEED, cw0=1 << 30, msg_prec=lx.MSG_F32, m=m)
    print("coarse FP32 sweep:", [(x, f"{b:.3g}") for x, b in pts])
    assert br is not None, "no bracket of BER 1e-4 on the grid"
    fine = [round(br[0] - 0.2 + 0.1 * i, 2) for i in range(7)]
    curves = {}
    for name, prec in [("fp32", lx.MSG_F32), ("fp16", lx.MSG_F16), ("fix6", lx.MSG_FIX6)]:
        curves[name] = [(x, ber.ber_point(code, x, codewords=N, seed=SEED, cw0=0, msg_prec=prec, m=m)["ber"])
                        for x in fine]
    ocode = orc.Code(1, 384, punct_cols=2)

    def oracle_ber(x):
        c = orc.sim(ocode, seed=SEED, cw0=0, B=N, ebn0_db=x, m=m, demap_method=orc.DEMAP_MAXLOG,
                    algo=orc.ALGO_MINSUM, iters=20, prec=0, store=orc.STORE_NATIVE, offset=0.5, clamp=20.0,
                    nthreads=os.cpu_count())
        return c[1] / c[0]

    # FP64 oracle at the points around the FP32 crossing, widened until it brackets its own crossing
    i = next(j for j in range(len(fine) - 1) if curves["fp32"][j][1] >= 1e-4 > curves["fp32"][j + 1][1])
    lo, hi = i, i + 1
    o = {fine[lo]: oracle_ber(fine[lo]), fine[hi]: oracle_ber(fine[hi])}
    while o[fine[lo]] < 1e-4 and lo > 0:
        lo -= 1
        o[fine[lo]] = oracle_ber(fine[lo])
    while o[fine[hi]] >= 1e-4 and hi < len(fine) - 1:
        hi += 1
        o[fine[hi]] = oracle_ber(fine[hi])
    curves["fp64"] = sorted(o.items())
    cross = {k: ber.crossing(v) for k, v in curves.items()}
    print("BER points:", {k: [(x, f"{b:.3g}") for x, b in v] for k, v in curves.items()})
    print("Eb/N0 at BER 1e-4:", {k: (None if v is None else round(v, 4)) for k, v in cross.items()})
    print("shift vs FP64 (dB):", {k: round(cross[k] - cross["fp64"], 4) for k in ("fp32", "fp16", "fix6")
                                  if cross[k] is not None and cross["fp64"] is not None})
    assert cross["fp64"] is not None and cross["fp32"] is not None and cross["fp16"] is not None
    assert abs(cross["fp32"] - cross["fp64"]) <= 0.05
    assert abs(cross["fp16"] - cross["fp64"]) <= 0.05
