"""One persistent launch over a batch that mixes codes (ldpc_bp_decode_mixed).

Each group's outputs (APP LLRs, hard decisions, iteration counts) must equal
ldpc_bp_decode on that group alone, bit for bit, and the FP32-replay oracle on
a sampled group; groups span both base-graph shapes, lifting sizes 8..384,
truncated rates, ragged sizes and an empty group.
"""
import numpy as np
import pytest

from tests import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GROUPS = [
    # (bg, Z, rows_kept, punct, B)
    (1, 384, 0, 2, 7),
    (2, 64, 0, 2, 37),
    (1, 16, 13, 2, 100),
    (2, 128, 7, 2, 9),
    (1, 256, 24, 2, 5),
    (2, 8, 0, 0, 130),
    (2, 32, 4, 2, 0),
]


@pytest.fixture(scope="module")
def lx():
    import paper_2203_11854_gb300 as lx
    assert torch.cuda.is_available()
    lx.load_library()
    return lx


def build_groups(lx, orc, seed=3):
    out = []
    for i, (bg, Z, rk, punct, B) in enumerate(GROUPS):
        code = lx.qc_ldpc_build(bg, Z, rows_kept=rk, punct_cols=punct)
        cw = np.zeros((B, code.n), dtype=np.uint8)
        if 0 < B and Z <= 64:  # real codewords where the oracle encoder is quick
            ocode = orc.Code(bg, Z, rows_kept=rk, punct_cols=punct)
            cw = ocode.encoder.encode(inputs.info_bits(seed + i, B, ocode.k))
        L = inputs.gaussian_llrs(cw, 2.6, seed + 10 * i)
        L_tx = np.ascontiguousarray(L[:, code.p0:code.p0 + code.n_tx])
        out.append((code, torch.from_numpy(L_tx).cuda()))
    return out


@pytest.mark.parametrize("algo,prec", [(0, 1), (0, 0), (0, 2), (1, 0), (1, 1)])
def test_mixed_equals_per_group(lx, orc, algo, prec):
    groups = build_groups(lx, orc)
    res = lx.ldpc_bp_decode_mixed(groups, algo=algo, iters=12, msg_prec=prec, early_stop=True, llr_out=True)
    stopped = 0
    for (code, llr), (lo, bits, its) in zip(groups, res):
        ref = lx.ldpc_bp_decode(code, llr, algo=algo, iters=12, msg_prec=prec, early_stop=True, llr_out=True)
        assert torch.equal(lo, ref[0]) and torch.equal(bits, ref[1]) and torch.equal(its, ref[2])
        stopped += int((its < 12).sum()) if its.numel() else 0
    assert stopped > 0
    assert lx.ldpcx_sync_status()[0] == 0


@pytest.mark.parametrize("cap", [1, 3, 8])
def test_mixed_work_item_cap_keeps_results(lx, orc, cap):
    """The tuned knob (codewords per work item) changes only how the batch is split into items."""
    groups = build_groups(lx, orc)
    ref = lx.ldpc_bp_decode_mixed(groups, algo=0, iters=12, msg_prec=1, early_stop=True, llr_out=True)
    try:
        lx.ldpcx_tune_set(lx.TUNE_CW_PER_CTA, cap)
        got = lx.ldpc_bp_decode_mixed(groups, algo=0, iters=12, msg_prec=1, early_stop=True, llr_out=True)
    finally:
        lx.ldpcx_tune_set(lx.TUNE_CW_PER_CTA, 0)
    for r, g in zip(ref, got):
        assert all(torch.equal(a, b) for a, b in zip(r, g) if a is not None)


def test_mixed_autotune(lx, orc, tmp_path):
    from paper_2203_11854_gb300 import autotune
    groups = build_groups(lx, orc)
    path = str(tmp_path / "tune.json")
    res = autotune.tune_mixed(groups, algo=0, msg_prec=1, iters=12, early_stop=True, cache_path=path,
                              candidates=(0, 4, 1))
    assert {t["cw_per_cta"] for t in res["timings"]} == {0, 4, 1}
    try:
        best = autotune.apply_mixed(groups, algo=0, msg_prec=1, iters=12, early_stop=True, cache_path=path)
        assert best == res["best"] and lx.ldpcx_tune_get(lx.TUNE_CW_PER_CTA) == best["cw_per_cta"]
    finally:
        lx.ldpcx_tune_set(lx.TUNE_CW_PER_CTA, 0)


def test_mixed_group_against_oracle(lx, orc):
    groups = build_groups(lx, orc)
    res = lx.ldpc_bp_decode_mixed(groups, algo=0, iters=12, msg_prec=1, early_stop=True, llr_out=True)
    code, llr = groups[2]
    bg, Z, rk, punct, B = GROUPS[2]
    ocode = orc.Code(bg, Z, rows_kept=rk, punct_cols=punct)
    app, hard, its = orc.decode(ocode.graph, orc.place_llr(llr.cpu().numpy().astype(np.float64), ocode.p0, ocode.n),
                                algo=0, iters=12, prec=1, store=1, early_stop=True)
    assert np.array_equal(res[2][0].cpu().numpy(), app.astype(np.float32))
    assert np.array_equal(res[2][2].cpu().numpy(), its)


@pytest.mark.parametrize("prec", [0, 1])
def test_mixed_spa_group_against_oracle(lx, orc, prec):
    """Layered sum-product in the mixed launch (FP32 and FP16 messages) against the FP64 oracle on one
    group, element by element within 1e-3 relative (absolute below |LLR| = 1) after clamping to +-20."""
    groups = build_groups(lx, orc)
    res = lx.ldpc_bp_decode_mixed(groups, algo=1, iters=12, msg_prec=prec, early_stop=False, llr_out=True)
    for gi in (1, 2):
        code, llr = groups[gi]
        bg, Z, rk, punct, B = GROUPS[gi]
        ocode = orc.Code(bg, Z, rows_kept=rk, punct_cols=punct)
        app, _, _ = orc.decode(ocode.graph, orc.place_llr(llr.cpu().numpy().astype(np.float64), ocode.p0, ocode.n),
                               algo=1, iters=12, store=orc.STORE_F16 if prec == 1 else orc.STORE_NATIVE)
        g = np.clip(res[gi][0].cpu().numpy().astype(np.float64), -20, 20)
        r = np.clip(app, -20, 20)
        err = np.abs(g - r) / np.maximum(np.abs(r), 1.0)
        assert (err <= 1e-3).all(), f"group {gi}: max scaled error {err.max():.3g}"


def test_mixed_rejects_flooding(lx, orc):
    groups = build_groups(lx, orc)
    with pytest.raises(lx.LdpcxError):
        lx.ldpc_bp_decode_mixed(groups, algo=lx.FLOOD_SPA, iters=5, msg_prec=0)
