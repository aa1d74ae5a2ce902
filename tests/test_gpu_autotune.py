"""Autotuner: every candidate knob setting gives identical outputs; the best is cached and applied."""
import json

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_tune_cache_apply(tmp_path):
    import paper_2203_11854_gb300 as lx
    from paper_2203_11854_gb300 import autotune
    assert torch.cuda.is_available()
    lx.load_library()
    cache = str(tmp_path / "tune.json")
    for bg, Z, prec in [(2, 64, lx.MSG_F16), (1, 384, lx.MSG_F32)]:
        code = lx.qc_ldpc_build(bg, Z, punct_cols=2 if bg == 1 else 0)
        res = autotune.tune(code, B=256, algo=lx.LAYERED_MINSUM, msg_prec=prec, iters=8, cache_path=cache)
        assert len(res["timings"]) >= 2 and res["best"]["ms"] > 0
        # check-node state: one and two check nodes per thread are both candidates
        assert {t["zpt"] for t in res["timings"]} == {0, 2}
        assert lx.ldpcx_tune_get(lx.TUNE_L2_PREFETCH) == 0 and lx.ldpcx_tune_get(lx.TUNE_CW_PER_CTA) == 0
        assert lx.ldpcx_tune_get(lx.TUNE_ZPT) == 0
        best = autotune.apply(code, algo=lx.LAYERED_MINSUM, msg_prec=prec, iters=8, cache_path=cache)
        assert best is not None
        assert lx.ldpcx_tune_get(lx.TUNE_L2_PREFETCH) == best["l2_prefetch"]
        assert lx.ldpcx_tune_get(lx.TUNE_CW_PER_CTA) == best["cw_per_cta"]
        assert lx.ldpcx_tune_get(lx.TUNE_ZPT) == best["zpt"]
        for key in (lx.TUNE_L2_PREFETCH, lx.TUNE_CW_PER_CTA, lx.TUNE_ZPT):
            lx.ldpcx_tune_set(key, 0)
    assert len(json.load(open(cache))) == 2
