"""Codes from caller-supplied base matrices and alist files (host logic, no
GPU): the alist text the library writes against a parity-check matrix built
here independently (numpy rolls of identities, and the oracle's lifted
graph); the library's alist parser against alist text written here from such
a matrix (padded and unpadded lines); malformed input; argument checks of
qc_ldpc_build_base; and the encodability test against a GF(2) rank computed
here."""
import numpy as np
import pytest

from tests import inputs


@pytest.fixture(scope="module")
def lx():
    import paper_2203_11854_gb300 as lx
    lx.load_library()
    return lx


def dense_from_base(S, Z):
    # block (r, c) with shift s: ones at (r Z + z, c Z + (z + s) mod Z), i.e. the identity rolled by s columns
    rows, cols = S.shape
    H = np.zeros((rows * Z, cols * Z), dtype=np.uint8)
    eye = np.eye(Z, dtype=np.uint8)
    for r in range(rows):
        for c in range(cols):
            if S[r, c] >= 0:
                H[r * Z:(r + 1) * Z, c * Z:(c + 1) * Z] = np.roll(eye, int(S[r, c]), axis=1)
    return H


def alist_text(H, pad=True):
    M, N = H.shape
    cw, rw = H.sum(axis=0), H.sum(axis=1)
    mc, mr = int(cw.max()), int(rw.max())
    out = [f"{N} {M}", f"{mc} {mr}", " ".join(map(str, cw)), " ".join(map(str, rw))]
    for j in range(N):
        idx = list(np.nonzero(H[:, j])[0] + 1) + ([0] * (mc - int(cw[j])) if pad else [])
        out.append(" ".join(map(str, idx)))
    for i in range(M):
        idx = list(np.nonzero(H[i])[0] + 1) + ([0] * (mr - int(rw[i])) if pad else [])
        out.append(" ".join(map(str, idx)))
    return "\n".join(out) + "\n"


def dense_from_alist(text):
    lines = [list(map(int, ln.split())) for ln in text.splitlines() if ln.strip()]
    N, M = lines[0]
    H = np.zeros((M, N), dtype=np.uint8)
    for i in range(M):
        for v in lines[4 + N + i]:
            if v:
                H[i, v - 1] = 1
    Hc = np.zeros_like(H)
    for j in range(N):
        for v in lines[4 + j]:
            if v:
                Hc[v - 1, j] = 1
    assert np.array_equal(H, Hc)
    assert list(H.sum(axis=0)) == lines[2] and list(H.sum(axis=1)) == lines[3]
    return H


def gf2_rank(A):
    A = A.copy() % 2
    r = 0
    for c in range(A.shape[1]):
        piv = next((i for i in range(r, A.shape[0]) if A[i, c]), None)
        if piv is None:
            continue
        A[[r, piv]] = A[[piv, r]]
        for i in range(A.shape[0]):
            if i != r and A[i, c]:
                A[i] ^= A[r]
        r += 1
    return r


def random_base(seed, Z, kb, rows, core="random"):
    """A base matrix with the transmitter's structure: core rows 0..3 over the systematic and four core parity
    columns, extension row r with its own parity column kb + r (random shift) and blocks among columns < kb + 4."""
    g = inputs.rng(seed)
    cols = kb + rows
    S = -np.ones((rows, cols), dtype=np.int16)
    for r in range(4):
        for c in g.choice(kb, size=max(2, kb // 2), replace=False):
            S[r, c] = g.integers(Z)
        if core == "random":
            for j in g.choice(4, size=2 + g.integers(2), replace=False):
                S[r, kb + j] = g.integers(Z)
    if core == "dual":
        for (r, j), s in {(0, 0): 1, (0, 1): 0, (1, 0): 0, (1, 1): 0, (1, 2): 0, (2, 2): 0, (2, 3): 0,
                          (3, 0): 1, (3, 3): 0}.items():
            S[r, kb + j] = s
    for r in range(4, rows):
        for c in g.choice(kb + 4, size=3, replace=False):
            S[r, c] = g.integers(Z)
        S[r, kb + r] = g.integers(Z)
    return S


def test_alist_export_matches_independent_matrix(lx, orc):
    code = lx.qc_ldpc_build(2, 8)
    S = code.base()
    H = dense_from_alist(lx.qc_ldpc_alist(code))
    assert np.array_equal(H, dense_from_base(S, 8))
    assert np.array_equal(H, orc.Graph(S, 8).dense())


@pytest.mark.parametrize("pad", [True, False])
@pytest.mark.parametrize("Z,kb,rows", [(5, 6, 7), (16, 8, 10), (3, 4, 4)])
def test_alist_import(lx, pad, Z, kb, rows):
    S = random_base(10 * Z + rows, Z, kb, rows)
    S2 = lx.qc_alist_parse(alist_text(dense_from_base(S, Z), pad=pad), Z)
    assert np.array_equal(S2, S)


def test_alist_round_trip_of_user_code(lx):
    S = random_base(3, 12, 6, 9)
    code = lx.qc_ldpc_build_base(S, 12, 6)
    assert np.array_equal(lx.qc_alist_parse(lx.qc_ldpc_alist(code), 12), S)


def test_alist_rejects_malformed(lx):
    S = random_base(4, 6, 4, 5)
    H = dense_from_base(S, 6)
    good = alist_text(H)
    assert lx.qc_alist_parse(good, 6).shape == S.shape
    with pytest.raises(lx.LdpcxError):
        lx.qc_alist_parse(good, 4)  # N, M not multiples of 4
    Hb = H.copy()  # one block no longer a shifted identity
    r, c = np.argwhere(Hb[:6, :6 * S.shape[1]])[0]
    Hb[r, c] = 0
    Hb[r, (c + 1) % Hb.shape[1]] ^= 1
    with pytest.raises(lx.LdpcxError):
        lx.qc_alist_parse(alist_text(Hb), 6)
    lines = good.splitlines()
    lines[4] = lines[4].replace(lines[4].split()[0], str(int(lines[4].split()[0]) % H.shape[0] + 1), 1)
    with pytest.raises(lx.LdpcxError):  # column list disagrees with the row lists
        lx.qc_alist_parse("\n".join(lines) + "\n", 6)
    with pytest.raises(lx.LdpcxError):
        lx.qc_alist_parse(good.replace("\n", "\nx ", 1), 6)
    with pytest.raises(lx.LdpcxError):
        lx.qc_alist_parse("\n".join(good.splitlines()[:-1]) + "\n", 6)  # a row list missing


def test_build_base_argument_checks(lx):
    S = random_base(5, 8, 6, 6)
    lx.qc_ldpc_build_base(S, 8, 6)
    bad = S.copy()
    bad[0, np.argmax(bad[0] >= 0)] = 8  # shift >= Z
    for args in [(bad, 8, 6), (S, 1, 6), (S, 8, S.shape[1]), (S, 8, 0), (S, 385, 6)]:
        with pytest.raises(lx.LdpcxError):
            lx.qc_ldpc_build_base(*args)
    one = S.copy()
    one[2] = -1
    one[2, 0] = 3  # a check row of one block
    with pytest.raises(lx.LdpcxError):
        lx.qc_ldpc_build_base(one, 8, 6)
    with pytest.raises(lx.LdpcxError):
        lx.qc_ldpc_build_base(S, 8, 6, punct_cols=7)


def test_seeded_matrix_as_user_matrix(lx):
    for bg, Z, rk in [(1, 16, 0), (2, 24, 9)]:
        c = lx.qc_ldpc_build(bg, Z, rows_kept=rk, punct_cols=2)
        u = lx.qc_ldpc_build_base(c.base(), Z, c.kb, punct_cols=2)
        for f in ("rows", "cols", "kb", "nnz", "max_row_deg", "n", "k", "n_tx", "p0", "edges", "encodable"):
            assert getattr(u, f) == getattr(c, f), f
        assert u.encodable == 1


@pytest.mark.parametrize("seed", range(8))
def test_encodable_matches_core_rank(lx, seed):
    Z, kb, rows = 6, 5, 7
    S = random_base(100 + seed, Z, kb, rows)
    core = dense_from_base(S[:4, kb:kb + 4], Z)
    code = lx.qc_ldpc_build_base(S, Z, kb)
    assert code.encodable == int(gf2_rank(core) == 4 * Z)


def test_not_encodable_structures(lx):
    S = random_base(7, 8, 6, 8, core="dual")
    assert lx.qc_ldpc_build_base(S, 8, 6).encodable == 1
    later = S.copy()
    later[5, 6 + 7] = 2  # extension row 5 reads the parity column of row 7
    assert lx.qc_ldpc_build_base(later, 8, 6).encodable == 0
    core_ext = S.copy()
    core_ext[1, 6 + 5] = 0  # a core row reads an extension parity column
    assert lx.qc_ldpc_build_base(core_ext, 8, 6).encodable == 0
    singular = S.copy()
    singular[1, 6:10] = singular[0, 6:10]
    singular[2, 6:10] = -1  # rows 0 and 1 of the core equal, row 2 empty: singular
    singular[2, 6:8] = 0
    singular[2, 8:10] = -1
    assert lx.qc_ldpc_build_base(singular, 8, 6).encodable == 0
    wide = np.concatenate([S, S[:, :1]], axis=1)  # cols != kb + rows
    assert lx.qc_ldpc_build_base(wide, 8, 6).encodable == 0
