"""Pins for the oracle's belief-propagation decoders.

* Sum-product on a cycle-free Tanner graph equals brute-force bitwise MAP.
* One check node of degree d: sum-product equals the tanh rule, min-sum
  (offset 0) equals brute-force max-log MAP over the check's configurations.
* Noiseless decoding returns the codeword after one iteration (early stop).
* Special cases: unit weights equal unweighted flooding; offset-0 min-sum is
  invariant to positive scaling of the LLRs; layered and flooding sum-product
  agree at high SNR; binary16 and 6-bit message stores against numpy.
* Statistical invariant: bit error rate does not depend on the codeword.
"""
import itertools
import math

import numpy as np
import pytest

# a cycle-free Tanner graph: 10 variables, 5 checks, 14 edges, connected
TREE_H = np.zeros((5, 10), dtype=np.uint8)
for c, vs in enumerate([(0, 1, 2), (2, 3, 4), (4, 5, 6), (1, 7), (6, 8, 9)]):
    TREE_H[c, list(vs)] = 1


@pytest.mark.parametrize("schedule", [0, 1])
def test_spa_on_tree_equals_bitwise_map(orc, schedule):
    g = orc.Graph.from_dense(TREE_H)
    rng = np.random.default_rng(5)
    for trial in range(5):
        L = rng.normal(scale=2.0, size=10)
        ref = orc.bitwise_map(TREE_H, L)
        app, _, _ = orc.decode(g, L[None], algo=orc.ALGO_SPA, schedule=schedule, iters=12, clamp=50.0)
        assert np.allclose(app[0], ref, rtol=1e-9, atol=1e-9)


def test_tree_layers_as_groups(orc):
    # two layers, each a set of checks touching disjoint variables
    H = TREE_H[[0, 2, 1, 3, 4]]
    g = orc.Graph.from_dense(H, layers=[0, 2, 5])
    L = np.random.default_rng(2).normal(size=10)
    app, _, _ = orc.decode(g, L[None], algo=orc.ALGO_SPA, schedule=0, iters=12, clamp=50.0)
    assert np.allclose(app[0], orc.bitwise_map(H, L), rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("d", [2, 3, 6, 19])
def test_single_parity_check(orc, d):
    H = np.ones((1, d), dtype=np.uint8)
    g = orc.Graph.from_dense(H)
    rng = np.random.default_rng(d)
    L = rng.normal(scale=3.0, size=d)
    # sum-product: extrinsic = 2 atanh(prod_{i != j} tanh(L_i / 2))
    app, _, _ = orc.decode(g, L[None], algo=orc.ALGO_SPA, iters=1, clamp=50.0)
    for j in range(d):
        others = np.delete(L, j)
        ext = 2 * math.atanh(np.prod(np.tanh(others / 2)))
        assert app[0, j] - L[j] == pytest.approx(ext, rel=1e-10, abs=1e-12)
    # min-sum, offset 0: extrinsic = max-log MAP of the check over the other bits
    app, _, _ = orc.decode(g, L[None], algo=orc.ALGO_MINSUM, iters=1, offset=0.0, clamp=50.0)
    for j in range(d):
        best = {0: -np.inf, 1: -np.inf}
        others = [i for i in range(d) if i != j]
        for bits in itertools.product([0, 1], repeat=d - 1):
            cj = sum(bits) % 2  # even parity fixes c_j
            met = -sum(b * L[i] for b, i in zip(bits, others))
            best[cj] = max(best[cj], met)
        assert app[0, j] - L[j] == pytest.approx(best[0] - best[1], abs=1e-12)
    # offset beta shrinks the magnitude by beta, floored at zero
    beta = 0.75
    app_b, _, _ = orc.decode(g, L[None], algo=orc.ALGO_MINSUM, iters=1, offset=beta, clamp=50.0)
    ext0 = app[0] - L
    extb = app_b[0] - L
    assert np.allclose(np.abs(extb), np.maximum(np.abs(ext0) - beta, 0.0), atol=1e-12)
    assert np.all((np.sign(extb) == np.sign(ext0)) | (extb == 0))


def test_minsum_ties_use_the_same_minimum(orc):
    H = np.ones((1, 4), dtype=np.uint8)
    g = orc.Graph.from_dense(H)
    L = np.array([1.5, -1.5, 3.0, 4.0])
    app, _, _ = orc.decode(g, L[None], algo=orc.ALGO_MINSUM, iters=1, offset=0.0)
    ext = app[0] - L
    assert ext.tolist() == [-1.5, 1.5, -1.5, -1.5]


ALL_VARIANTS = [
    dict(algo=0, schedule=0, store=0), dict(algo=0, schedule=0, store=1), dict(algo=0, schedule=0, store=2),
    dict(algo=1, schedule=0, store=0), dict(algo=1, schedule=1, store=0), dict(algo=0, schedule=1, store=0),
    dict(algo=0, schedule=0, store=0, prec=1), dict(algo=1, schedule=0, store=1, prec=1),
]


@pytest.mark.parametrize("bg,Z", [(2, 8), (1, 16)])
@pytest.mark.parametrize("var", ALL_VARIANTS)
def test_noiseless_decode(orc, bg, Z, var):
    code = orc.Code(bg, Z)
    u = orc.source_bits(3, 0, 4, code.k)
    cw = code.encoder.encode(u)
    L = 20.0 * (1.0 - 2.0 * cw)
    app, hard, its = orc.decode(code.graph, L, iters=10, early_stop=True, **var)
    assert (hard == cw).all()
    assert (its == 1).all()
    assert np.all(np.sign(app) == 1 - 2.0 * cw)


def test_single_error_corrected(orc):
    code = orc.Code(2, 8)
    u = orc.source_bits(4, 0, 1, code.k)
    cw = code.encoder.encode(u)
    L = 6.0 * (1.0 - 2.0 * cw)
    for v in [0, 17, 100, 415]:
        Lf = L.copy()
        Lf[0, v] = -0.5 * Lf[0, v]  # weak wrong-sign LLR
        for algo in (0, 1):
            _, hard, its = orc.decode(code.graph, Lf, algo=algo, iters=20, early_stop=True)
            assert (hard == cw).all()
            assert its[0] <= 3


def test_unit_weights_equal_plain_flooding(orc):
    code = orc.Code(2, 8)
    rng = np.random.default_rng(9)
    L = rng.normal(loc=1.0, scale=2.0, size=(6, code.n))
    for algo in (0, 1):
        w = np.ones((10, code.graph.n_cls))
        a1, h1, _ = orc.decode(code.graph, L, algo=algo, schedule=1, iters=10, weights=w)
        a0, h0, _ = orc.decode(code.graph, L, algo=algo, schedule=1, iters=10)
        assert np.array_equal(a1, a0)
        # non-unit weights do change the result
        a2, _, _ = orc.decode(code.graph, L, algo=algo, schedule=1, iters=10, weights=0.7 * w)
        assert not np.allclose(a2, a0)


def test_minsum_offset0_scale_invariance(orc):
    code = orc.Code(2, 8)
    rng = np.random.default_rng(4)
    L = rng.normal(loc=0.8, scale=1.5, size=(8, code.n))
    for schedule in (0, 1):
        a1, h1, _ = orc.decode(code.graph, L, schedule=schedule, offset=0.0, clamp=1e6, iters=15)
        a2, h2, _ = orc.decode(code.graph, 2.0 * L, schedule=schedule, offset=0.0, clamp=1e6, iters=15)
        assert np.array_equal(h1, h2)
        assert np.array_equal(2.0 * a1, a2)


def run_chain(orc, code, ebn0, m, seed, B, zero_codeword=False):
    u = orc.source_bits(seed, 0, B, code.k)
    if zero_codeword:
        u[:] = 0
    cw = code.encoder.encode(u)
    N0 = orc.n0_from_ebn0(ebn0, code.k, code.n_tx, m)
    x = orc.map_bits(cw, m, code.p0, code.n_tx)
    y = orc.awgn(x, m, N0, seed + 1, 0)
    ltx = orc.demap(y, m, N0, orc.DEMAP_EXACT)
    return u, cw, orc.place_llr(ltx, code.p0, code.n)


def test_layered_and_flooding_agree_at_high_snr(orc):
    code = orc.Code(2, 16)
    u, cw, L = run_chain(orc, code, 4.0, 2, 17, 40)
    _, hl, _ = orc.decode(code.graph, L, algo=1, schedule=0, iters=20)
    _, hf, _ = orc.decode(code.graph, L, algo=1, schedule=1, iters=20)
    assert np.array_equal(hl, hf)
    assert np.array_equal(hl, cw)


def test_fp32_replay_tracks_fp64(orc):
    code = orc.Code(2, 16)
    _, cw, L = run_chain(orc, code, 2.0, 2, 23, 40)
    a64, h64, _ = orc.decode(code.graph, L, iters=10)
    a32, h32, _ = orc.decode(code.graph, L, iters=10, prec=1)
    assert (h64 != h32).mean() < 1e-3
    # every FP32-replay value is a binary32 number
    assert np.array_equal(a32.astype(np.float32).astype(np.float64), a32)


def test_message_stores_against_numpy(orc):
    rng = np.random.default_rng(0)
    xs = np.concatenate([rng.normal(scale=5, size=2000), rng.uniform(-1e-4, 1e-4, size=200),
                         [0.0, -0.0, 20.0, -20.0, 1.0 + 2 ** -11, 1.0 + 3 * 2 ** -11, 2 ** -25, 3 * 2 ** -25]])
    for x in xs:
        assert orc.to_half(x) == float(np.float64(x).astype(np.float16))
        x32 = float(np.float32(x))
        assert orc.to_half(x32) == float(np.float32(x32).astype(np.float16))
    # 6-bit fixed point, step 0.5: nearest multiple (ties to even step), saturated at 31 steps
    cases = {0.0: 0.0, 0.24: 0.0, 0.25: 0.0, 0.26: 0.5, 0.75: 1.0, 1.25: 1.0, -0.75: -1.0, 15.4: 15.5,
             16.0: 15.5, -20.0: -15.5, 7.3: 7.5}
    for x, q in cases.items():
        assert orc.to_fix6(x) == q


def test_phi(orc):
    for x in [1e-6, 0.01, 0.5, 1.0, 3.0, 10.0]:
        assert orc.phi(x) == pytest.approx(-math.log(math.tanh(x / 2)), rel=1e-12)
        assert orc.phi(orc.phi(x)) == pytest.approx(x, rel=1e-9)
    assert orc.phi(20.0) == pytest.approx(2 * math.exp(-20.0), rel=1e-8)


def test_stored_messages_are_rounded(orc):
    # decoding with the binary16 store must reach only APP values T + R with R a
    # binary16 number; check on a single check node where APP - L is the message
    H = np.ones((1, 5), dtype=np.uint8)
    g = orc.Graph.from_dense(H)
    L = np.array([1.1, -2.3, 3.7, 0.9, -4.1])
    for store, check in [(1, lambda r: float(np.float64(r).astype(np.float16)) == r),
                         (2, lambda r: (r * 2).is_integer() and abs(r) <= 15.5)]:
        for algo in (0, 1):
            app, _, _ = orc.decode(g, L[None], algo=algo, iters=1, store=store)
            for r in app[0] - L:
                assert check(round(r, 12)) or check(r)


def test_ber_is_codeword_independent(orc):
    code = orc.Code(2, 8)
    B = 600
    res = []
    for zero in (False, True):
        u, cw, L = run_chain(orc, code, 1.5, 2, 41, B, zero_codeword=zero)
        _, hard, _ = orc.decode(code.graph, L, iters=10)
        res.append(int((hard[:, :code.k] != u).sum()))
    n = B * code.k
    p = (res[0] + res[1]) / (2 * n)
    sd = math.sqrt(2 * n * p * (1 - p))
    assert p > 1e-3  # the comparison is not vacuous
    assert abs(res[0] - res[1]) < 6 * sd + 5


def test_early_stop_counts(orc):
    code = orc.Code(2, 8)
    _, cw, L = run_chain(orc, code, 3.0, 2, 43, 50)
    app, hard, its = orc.decode(code.graph, L, iters=20, early_stop=True)
    synd = code.graph.syndrome(hard)
    for b in range(50):
        if its[b] < 20:
            assert not synd[b].any()
    # without early stop the count is the iteration limit
    _, _, its2 = orc.decode(code.graph, L, iters=20)
    assert (its2 == 20).all()


def test_sim_chain_counts(orc):
    code = orc.Code(2, 8)
    counts = orc.sim(code, seed=5, cw0=0, B=64, ebn0_db=2.0, m=2, demap_method=orc.DEMAP_EXACT,
                     nthreads=3)
    u, cw, L = run_chain_sim_layout(orc, code, 2.0, 2, 5, 64)
    _, hard, its = orc.decode(code.graph, L, iters=20)
    errs = (hard[:, :code.k] != u).sum(axis=1)
    assert counts.tolist() == [64 * code.k, int(errs.sum()), 64, int((errs > 0).sum()), int(its.sum())]
    # thread count does not change results
    c1 = orc.sim(code, seed=5, cw0=0, B=64, ebn0_db=2.0, m=2, demap_method=orc.DEMAP_EXACT, nthreads=1)
    assert counts.tolist() == c1.tolist()


def run_chain_sim_layout(orc, code, ebn0, m, seed, B):
    # the sim draws source bits and noise from the same seed
    u = orc.source_bits(seed, 0, B, code.k)
    cw = code.encoder.encode(u)
    N0 = orc.n0_from_ebn0(ebn0, code.k, code.n_tx, m)
    y = orc.awgn(orc.map_bits(cw, m, code.p0, code.n_tx), m, N0, seed, 0)
    ltx = orc.demap(y, m, N0, orc.DEMAP_EXACT)
    return u, cw, orc.place_llr(ltx, code.p0, code.n)
