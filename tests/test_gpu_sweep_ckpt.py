"""Checkpoint / resume of the Monte-Carlo sweep (sim_run with ckpt_path).

A sweep run in slices (max_points), each call restoring the previous call's
checkpoint, must give the uninterrupted sweep's int64 counts bit for bit --
also when a point ends early on min_bit_errors (so the codeword index where
the next point starts depends on the batches actually run), when slices
switch between graph and eager mode, and when the sweep stops on stop_ber.
A finished sweep returns its saved counts; a checkpoint of another sweep is
refused."""
import json

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lx():
    import paper_2203_11854_gb300 as lx
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    lx.load_library()
    return lx


GRID = [1.0, 1.5, 2.0, 2.5, 3.0]
KW = dict(m=4, batch=384, max_batches=4, min_bit_errors=400, iters=12, early_stop=True, seed=0x5EED, cw0=77)


def test_sliced_sweep_equals_uninterrupted(lx, tmp_path):
    code = lx.qc_ldpc_build(2, 64, punct_cols=2)
    ref = lx.sim_run(code, GRID, use_graph=True, **KW)
    assert len(ref) == len(GRID)
    # min_bit_errors ends some points before max_batches: the next point's first codeword moves with it
    assert len({p["blocks"] for p in ref}) > 1
    path = str(tmp_path / "sweep.json")
    got = lx.sim_run(code, GRID, ckpt_path=path, max_points=1, use_graph=True, **KW)
    assert len(got) == 1 and got == ref[:1]
    state = json.load(open(path))
    assert state["next_point"] == 1 and state["finished"] == 0 and len(state["points"]) == 1
    assert state["next_cw"] == KW["cw0"] + ref[0]["blocks"]
    got = lx.sim_run(code, GRID, ckpt_path=path, max_points=2, use_graph=False, **KW)  # eager slice
    assert got == ref[:3]
    got = lx.sim_run(code, GRID, ckpt_path=path, use_graph=True, **KW)
    assert got == ref
    state = json.load(open(path))
    assert state["finished"] == 1 and state["next_point"] == len(GRID)
    assert [p["bit_errors"] for p in state["points"]] == [p["bit_errors"] for p in ref]
    # a finished sweep returns its saved counts
    assert lx.sim_run(code, GRID, ckpt_path=path, **KW) == ref


def test_resume_after_stop_ber(lx, tmp_path):
    code = lx.qc_ldpc_build(2, 64, punct_cols=2)
    kw = dict(KW, stop_ber=2e-3, min_bit_errors=0, max_batches=2)
    grid = [1.0, 2.0, 3.0, 4.0, 5.0, 6.0]
    ref = lx.sim_run(code, grid, **kw)
    assert len(ref) < len(grid)  # the sweep stopped early
    path = str(tmp_path / "stop.json")
    first = lx.sim_run(code, grid, ckpt_path=path, max_points=1, **kw)
    assert first == ref[:1]
    assert lx.sim_run(code, grid, ckpt_path=path, **kw) == ref
    assert json.load(open(path))["finished"] == 1
    assert lx.sim_run(code, grid, ckpt_path=path, **kw) == ref


def test_checkpoint_of_another_sweep_is_refused(lx, tmp_path):
    code = lx.qc_ldpc_build(2, 64, punct_cols=2)
    path = str(tmp_path / "a.json")
    lx.sim_run(code, GRID, ckpt_path=path, max_points=1, **KW)
    for change in (dict(seed=1), dict(batch=256), dict(iters=11), dict(cw0=0)):
        with pytest.raises(lx.LdpcxError, match="IO"):
            lx.sim_run(code, GRID, ckpt_path=path, **{**KW, **change})
    with pytest.raises(lx.LdpcxError, match="IO"):
        lx.sim_run(code, GRID[:-1], ckpt_path=path, **KW)
    other = lx.qc_ldpc_build(2, 64, punct_cols=2, seed=9)
    with pytest.raises(lx.LdpcxError, match="IO"):
        lx.sim_run(other, GRID, ckpt_path=path, **KW)
