"""FP64 CPU oracle for the QC-LDPC Monte-Carlo hot path (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package. The product
library (``paper_2203_11854_gb300``) never imports it, and the two share no
code: this package wraps ``ldpc_oracle.c`` (plain C, compiled with gcc) through
ctypes and numpy, and holds the CPU restatement of each step:

* seeded BG-shaped base matrices and their lifting (the paper's LDPC5GEncoder,
  Sec. III-B; the 3GPP tables are not available, so codes are seeded);
* a GF(2) Gauss-Jordan systematic encoder;
* Philox4x32-10 source bits and Box-Muller AWGN (BinarySource, AWGN, Listing 1);
* the Gray square-QAM mapper and the exact / max-log APP demapper
  (Constellation, Mapper, Demapper("app"), Listing 1);
* layered and flooding belief propagation, offset min-sum and sum-product
  (LDPC5GDecoder, "BP decoder and variants", Sec. III-B; min-sum BP as the
  custom CUDA op of Sec. IV-A);
* brute-force bitwise MAP for tiny codes, and integer error counting
  (compute_ber, Listing 1).

Everything is FP64 unless ``prec=1`` asks for the FP32 replay (each operation
of the check-node and variable-node updates rounded to binary32 in the same
order as the definition).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ldpc_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "polar_oracle.c")]
_LIB_PATH = os.path.join(_HERE, "libldpc_oracle.so")
_lib = None
_lock = threading.Lock()

ALGO_MINSUM, ALGO_SPA = 0, 1
SCHED_LAYERED, SCHED_FLOOD = 0, 1
STORE_NATIVE, STORE_F16, STORE_FIX6 = 0, 1, 2
DEMAP_EXACT, DEMAP_MAXLOG = 0, 1

_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
_i16p = np.ctypeslib.ndpointer(dtype=np.int16, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile ldpc_oracle.c and polar_oracle.c with gcc (no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB_PATH) or any(os.path.getmtime(_LIB_PATH) < os.path.getmtime(f)
                                                       for f in _SRCS):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call([
            "gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
            "-o", tmp, *_SRCS, "-lm", "-lpthread",
        ])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.orc_base_matrix.argtypes = [C.c_int, C.c_int, C.c_uint64, C.c_int, _i16p, _i32p]
            L.orc_lift.argtypes = [_i16p, C.c_int, C.c_int, C.c_int, _i32p, _i32p, _i32p, _i32p]
            L.orc_enc_prepare.argtypes = [_i16p, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int32)]
            L.orc_enc_prepare.restype = C.c_void_p
            L.orc_enc_free.argtypes = [C.c_void_p]
            L.orc_enc_encode.argtypes = [C.c_void_p, _u8p, C.c_int64, _u8p]
            L.orc_philox_many.argtypes = [C.c_int64, _u32p, _u32p, _u32p]
            L.orc_source_bits.argtypes = [C.c_uint64, C.c_uint64, C.c_int64, C.c_int, _u8p]
            L.orc_qam_scale.argtypes = [C.c_int]
            L.orc_qam_scale.restype = C.c_double
            L.orc_map.argtypes = [_u8p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int64, _f64p]
            L.orc_gauss_pair.argtypes = [C.c_uint32, C.c_uint32, C.POINTER(C.c_double), C.POINTER(C.c_double)]
            L.orc_awgn.argtypes = [_f64p, C.c_int64, C.c_int, C.c_int, _f64p, C.c_uint64, C.c_uint64, _f64p]
            L.orc_n0_from_ebn0.argtypes = [C.c_double, C.c_int, C.c_int, C.c_int]
            L.orc_n0_from_ebn0.restype = C.c_double
            L.orc_demap.argtypes = [_f64p, C.c_int64, C.c_int, C.c_int, _f64p, C.c_int, C.c_double, _f64p]
            L.orc_demap_prior.argtypes = [_f64p, C.c_int64, C.c_int, C.c_int, _f64p, C.c_int, C.c_double,
                                          C.c_void_p, C.c_int, _f64p]
            L.orc_apriori.argtypes = [_u8p, C.c_int64, C.c_int64, C.c_double, C.c_uint64, C.c_uint64, _f64p]
            L.orc_polar_bhatt.argtypes = [C.c_int, C.c_double, _f64p]
            L.orc_polar_info_set.argtypes = [C.c_int, C.c_double, C.c_int, _i32p, _u8p]
            L.orc_polar_encode.argtypes = [C.c_int, _u8p, _u8p]
            L.orc_polar_encode.restype = None
            L.orc_crc.argtypes = [_u8p, C.c_int, C.c_uint64, C.c_int, _u8p]
            L.orc_crc.restype = None
            L.orc_polar_scl.argtypes = [C.c_int, _f64p, C.c_int64, _u8p, _i32p, C.c_int, C.c_int, C.c_uint64,
                                        C.c_int, C.c_int, _u8p, _f64p]
            L.orc_demap_points.argtypes = [_f64p, C.c_int64, C.c_int, C.c_int, _f64p, _f64p, C.c_int, C.c_double,
                                           _f64p]
            L.orc_apriori.restype = None
            L.orc_place_llr.argtypes = [_f64p, C.c_int64, C.c_int, C.c_int, C.c_int, _f64p]
            L.orc_to_half.argtypes = [C.c_double]
            L.orc_to_half.restype = C.c_double
            L.orc_to_fix6.argtypes = [C.c_double]
            L.orc_to_fix6.restype = C.c_double
            L.orc_phi.argtypes = [C.c_double]
            L.orc_phi.restype = C.c_double
            L.orc_splitmix64_next.argtypes = [C.POINTER(C.c_uint64)]
            L.orc_splitmix64_next.restype = C.c_uint64
            L.orc_decode.argtypes = [
                C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                _i32p, _i32p, _i32p, _i32p,
                C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                C.c_double, C.c_double, C.c_void_p,
                _f64p, C.c_int64, _f64p, _u8p, _i32p, C.c_int,
            ]
            L.orc_bitwise_map.argtypes = [_u8p, C.c_int, C.c_int, _f64p, _f64p]
            L.orc_sim.argtypes = [
                C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                _i32p, _i32p, _i32p, _i32p,
                C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double,
                C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                C.c_uint64, C.c_uint64, C.c_int64, C.c_double, _i64p, C.c_int,
            ]
            _lib = L
    return _lib


def _check(st: int, what: str) -> None:
    if st < 0:
        raise RuntimeError(f"oracle {what} failed with status {st}")


# --------------------------------------------------------------------------- codes
def base_matrix(bg: int, Z: int, seed: int, rows_kept: int = 0) -> tuple[np.ndarray, int]:
    """Seeded BG-shaped base matrix S (rows x cols, -1 = zero block) and Kb."""
    S = np.zeros(46 * 68, dtype=np.int16)
    dims = np.zeros(3, dtype=np.int32)
    _check(lib().orc_base_matrix(bg, Z, seed, rows_kept, S, dims), "base_matrix")
    rows, cols, kb = (int(x) for x in dims)
    return S[: rows * cols].reshape(rows, cols).copy(), kb


class Graph:
    """Lifted Tanner graph: check nodes r*Z+z (layer r), edges in ascending base column."""

    def __init__(self, S: np.ndarray, Z: int):
        S = np.ascontiguousarray(S, dtype=np.int16)
        rows, cols = S.shape
        nnz = int((S >= 0).sum())
        self.S, self.Z, self.rows, self.cols, self.nnz = S, Z, rows, cols, nnz
        self.n, self.m, self.E = cols * Z, rows * Z, nnz * Z
        self.n_layers, self.n_cls = rows, nnz
        self.cn_ptr = np.zeros(self.m + 1, dtype=np.int32)
        self.edge_vn = np.zeros(self.E, dtype=np.int32)
        self.edge_cls = np.zeros(self.E, dtype=np.int32)
        self.layer_ptr = np.zeros(rows + 1, dtype=np.int32)
        e = lib().orc_lift(S.reshape(-1), rows, cols, Z, self.cn_ptr, self.edge_vn, self.edge_cls, self.layer_ptr)
        _check(e, "lift")
        assert e == self.E

    @classmethod
    def from_dense(cls_, H: np.ndarray, layers: list[int] | None = None) -> "Graph":
        """Graph of an arbitrary dense H (each check node its own layer unless given)."""
        g = cls_.__new__(cls_)
        H = np.asarray(H, dtype=np.uint8)
        m, n = H.shape
        g.S, g.Z, g.rows, g.cols = None, 1, m, n
        g.n, g.m = n, m
        vn, ptr = [], [0]
        for c in range(m):
            vn.extend(np.nonzero(H[c])[0].tolist())
            ptr.append(len(vn))
        g.E = len(vn)
        g.nnz = g.E
        g.cn_ptr = np.asarray(ptr, dtype=np.int32)
        g.edge_vn = np.asarray(vn, dtype=np.int32)
        g.edge_cls = np.arange(g.E, dtype=np.int32)
        g.n_cls = g.E
        if layers is None:
            layers = list(range(m + 1))
        g.layer_ptr = np.asarray(layers, dtype=np.int32)
        g.n_layers = len(layers) - 1
        return g

    def dense(self) -> np.ndarray:
        H = np.zeros((self.m, self.n), dtype=np.uint8)
        for c in range(self.m):
            H[c, self.edge_vn[self.cn_ptr[c]: self.cn_ptr[c + 1]]] ^= 1
        return H

    def syndrome(self, bits: np.ndarray) -> np.ndarray:
        """H c over GF(2) for bits [B, n] (uses the edge lists directly)."""
        bits = np.asarray(bits, dtype=np.uint8).reshape(-1, self.n)
        gathered = bits[:, self.edge_vn]
        out = np.zeros((bits.shape[0], self.m), dtype=np.uint8)
        for c in range(self.m):
            out[:, c] = np.bitwise_xor.reduce(gathered[:, self.cn_ptr[c]: self.cn_ptr[c + 1]], axis=1)
        return out


class Encoder:
    """Systematic encoder from GF(2) Gauss-Jordan elimination of [H_p | H_s]."""

    def __init__(self, S: np.ndarray, Kb: int, Z: int):
        S = np.ascontiguousarray(S, dtype=np.int16)
        rows, cols = S.shape
        st = C.c_int32(0)
        self._h = lib().orc_enc_prepare(S.reshape(-1), rows, cols, Kb, Z, C.byref(st))
        if st.value != 0 or not self._h:
            raise RuntimeError(f"oracle encoder preparation failed with status {st.value}")
        self.n, self.k = cols * Z, Kb * Z

    def encode(self, u: np.ndarray) -> np.ndarray:
        u = np.ascontiguousarray(u, dtype=np.uint8).reshape(-1, self.k)
        c = np.zeros((u.shape[0], self.n), dtype=np.uint8)
        _check(lib().orc_enc_encode(self._h, u, u.shape[0], c), "encode")
        return c

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_enc_free(h)
            self._h = None


# --------------------------------------------------------------------------- random draws
def philox(ctr: np.ndarray, key: tuple[int, int]) -> np.ndarray:
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    out = np.zeros_like(ctr)
    lib().orc_philox_many(ctr.shape[0], ctr, np.asarray(key, dtype=np.uint32), out)
    return out


def source_bits(seed: int, cw0: int, B: int, k: int) -> np.ndarray:
    u = np.zeros((B, k), dtype=np.uint8)
    lib().orc_source_bits(seed, cw0, B, k, u)
    return u


def gauss_pair(a: int, b: int) -> tuple[float, float]:
    g0, g1 = C.c_double(), C.c_double()
    lib().orc_gauss_pair(a, b, C.byref(g0), C.byref(g1))
    return g0.value, g1.value


# --------------------------------------------------------------------------- channel
def qam_scale(m: int) -> float:
    return float(lib().orc_qam_scale(m))


def map_bits(cw: np.ndarray, m: int, p0: int = 0, n_tx: int | None = None) -> np.ndarray:
    cw = np.ascontiguousarray(cw, dtype=np.uint8)
    B, n = cw.shape
    n_tx = n - p0 if n_tx is None else n_tx
    S = n_tx // m
    x = np.zeros((B, S) if m == 1 else (B, S, 2), dtype=np.float64)
    _check(lib().orc_map(cw, n, p0, n_tx, m, B, x.reshape(-1)), "map")
    return x


def awgn(x: np.ndarray, m: int, N0, seed: int, cw0: int) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    B, S = x.shape[0], x.shape[1]
    n0 = np.broadcast_to(np.asarray(N0, dtype=np.float64), (B,)).copy()
    y = np.zeros_like(x)
    lib().orc_awgn(x.reshape(-1), B, S, m, n0, seed, cw0, y.reshape(-1))
    return y


def n0_from_ebn0(ebn0_db: float, k: int, n_tx: int, m: int) -> float:
    return float(lib().orc_n0_from_ebn0(ebn0_db, k, n_tx, m))


def demap(y: np.ndarray, m: int, N0, method: int = DEMAP_EXACT, clamp: float = 20.0) -> np.ndarray:
    y = np.ascontiguousarray(y, dtype=np.float64)
    B, S = y.shape[0], y.shape[1]
    n0 = np.broadcast_to(np.asarray(N0, dtype=np.float64), (B,)).copy()
    llr = np.zeros((B, S * m), dtype=np.float64)
    _check(lib().orc_demap(y.reshape(-1), B, S, m, n0, method, clamp, llr.reshape(-1)), "demap")
    return llr


def demap_prior(y: np.ndarray, m: int, N0, prior=None, method: int = DEMAP_EXACT, clamp: float = 20.0,
                mode: int = 1) -> np.ndarray:
    """Demapper with a-priori LLRs (mode 0: a-posteriori, 1: extrinsic), full 2-D FP64 sums."""
    y = np.ascontiguousarray(y, dtype=np.float64)
    B, S = y.shape[0], y.shape[1]
    n0 = np.broadcast_to(np.asarray(N0, dtype=np.float64), (B,)).copy()
    llr = np.zeros((B, S * m), dtype=np.float64)
    pr = None if prior is None else np.ascontiguousarray(prior, dtype=np.float64).reshape(-1)
    _check(lib().orc_demap_prior(y.reshape(-1), B, S, m, n0, method, clamp,
                                 None if pr is None else pr.ctypes.data, mode, llr.reshape(-1)), "demap_prior")
    return llr


def demap_points(y: np.ndarray, m: int, N0, points: np.ndarray, method: int = DEMAP_EXACT,
                 clamp: float = 20.0) -> np.ndarray:
    """APP demapper over the constellation points [2^m, 2] (label of point l = l, MSB first), y [B, S, 2]."""
    y = np.ascontiguousarray(y, dtype=np.float64)
    B, S = y.shape[0], y.shape[1]
    n0 = np.broadcast_to(np.asarray(N0, dtype=np.float64), (B,)).copy()
    pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1)
    llr = np.zeros((B, S * m), dtype=np.float64)
    _check(lib().orc_demap_points(y.reshape(-1), B, S, m, n0, pts, method, clamp, llr.reshape(-1)),
           "demap_points")
    return llr


# ----------------------------------------------------------------- polar codes
def polar_bhatt(n: int, design_esn0_db: float) -> np.ndarray:
    z = np.zeros(1 << n, dtype=np.float64)
    _check(lib().orc_polar_bhatt(n, design_esn0_db, z), "polar_bhatt")
    return z


def polar_info_set(n: int, K: int, design_esn0_db: float):
    """(info indices ascending int32 [K], frozen mask uint8 [N])."""
    info = np.zeros(max(K, 1), dtype=np.int32)
    frozen = np.zeros(1 << n, dtype=np.uint8)
    _check(lib().orc_polar_info_set(n, design_esn0_db, K, info, frozen), "polar_info_set")
    return info[:K], frozen


def polar_encode(u: np.ndarray) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.uint8)
    out = np.zeros_like(u)
    n = int(np.log2(u.shape[-1]))
    for r in range(u.reshape(-1, u.shape[-1]).shape[0]):
        lib().orc_polar_encode(n, u.reshape(-1, u.shape[-1])[r], out.reshape(-1, u.shape[-1])[r])
    return out


def crc(bits: np.ndarray, g: int, r: int) -> np.ndarray:
    bits = np.ascontiguousarray(bits, dtype=np.uint8)
    out = np.zeros(r, dtype=np.uint8)
    lib().orc_crc(bits, bits.size, g, r, out)
    return out


def polar_scl(llr: np.ndarray, frozen: np.ndarray, info: np.ndarray, L: int, g: int = 0, r: int = 0,
              prec: int = 0):
    """(u_hat uint8 [B, N], path metric [B]) of CRC-aided SCL (L = 1: SC)."""
    llr = np.ascontiguousarray(llr, dtype=np.float64)
    B, N = llr.shape
    n = int(np.log2(N))
    uh = np.zeros((B, N), dtype=np.uint8)
    pm = np.zeros(B, dtype=np.float64)
    _check(lib().orc_polar_scl(n, llr.reshape(-1), B, np.ascontiguousarray(frozen, dtype=np.uint8),
                               np.ascontiguousarray(info, dtype=np.int32), len(info), L, g, r, prec,
                               uh.reshape(-1), pm), "polar_scl")
    return uh, pm


def qam_points(m: int) -> np.ndarray:
    """The Gray QAM of the mapper as points [2^m, 2], point l carrying label l (MSB first)."""
    P = 1 << m
    bits = ((np.arange(P)[:, None] >> (m - 1 - np.arange(m))[None, :]) & 1).astype(np.uint8)
    x = map_bits(bits, m)
    return np.ascontiguousarray(x[:, 0, :])


def apriori(bits: np.ndarray, sigma: float, seed: int, cw0: int) -> np.ndarray:
    """Consistent Gaussian a-priori LLRs of the unpacked bits [B, N] (Philox stream 2)."""
    bits = np.ascontiguousarray(bits, dtype=np.uint8)
    B, N = bits.shape
    out = np.zeros((B, N), dtype=np.float64)
    lib().orc_apriori(bits.reshape(-1), B, N, float(sigma), seed, cw0, out.reshape(-1))
    return out


def place_llr(llr_tx: np.ndarray, p0: int, n: int) -> np.ndarray:
    llr_tx = np.ascontiguousarray(llr_tx, dtype=np.float64)
    B, n_tx = llr_tx.shape
    out = np.zeros((B, n), dtype=np.float64)
    lib().orc_place_llr(llr_tx.reshape(-1), B, n_tx, p0, n, out.reshape(-1))
    return out


# --------------------------------------------------------------------------- decoding
def to_half(x: float) -> float:
    return float(lib().orc_to_half(float(x)))


def to_fix6(x: float) -> float:
    return float(lib().orc_to_fix6(float(x)))


def phi(x: float) -> float:
    return float(lib().orc_phi(float(x)))


def decode(g: Graph, llr: np.ndarray, *, algo: int = ALGO_MINSUM, schedule: int = SCHED_LAYERED,
           iters: int = 20, prec: int = 0, store: int = STORE_NATIVE, early_stop: bool = False,
           offset: float = 0.5, clamp: float = 20.0, weights: np.ndarray | None = None,
           nthreads: int | None = None):
    """Decode llr [B, n] (channel LLRs with punctured positions already 0).

    Returns (app [B, n] float64, hard [B, n] uint8, iters [B] int32).
    """
    llr = np.ascontiguousarray(llr, dtype=np.float64).reshape(-1, g.n)
    B = llr.shape[0]
    app = np.zeros((B, g.n), dtype=np.float64)
    hard = np.zeros((B, g.n), dtype=np.uint8)
    its = np.zeros(B, dtype=np.int32)
    wptr = None
    if weights is not None:
        weights = np.ascontiguousarray(weights, dtype=np.float64)
        assert weights.shape == (iters, g.n_cls)
        wptr = weights.ctypes.data
    nthreads = nthreads or min(os.cpu_count() or 1, max(1, B))
    st = lib().orc_decode(g.n, g.m, g.E, g.n_layers, g.n_cls, g.cn_ptr, g.edge_vn, g.edge_cls, g.layer_ptr,
                          algo, schedule, iters, prec, store, int(early_stop), offset, clamp, wptr,
                          llr.reshape(-1), B, app, hard, its, nthreads)
    _check(st, "decode")
    return app, hard, its


def bitwise_map(H: np.ndarray, L: np.ndarray) -> np.ndarray:
    H = np.ascontiguousarray(H, dtype=np.uint8)
    m, n = H.shape
    L = np.ascontiguousarray(L, dtype=np.float64)
    out = np.zeros(n, dtype=np.float64)
    _check(lib().orc_bitwise_map(H.reshape(-1), m, n, L, out), "bitwise_map")
    return out


class Code:
    """A seeded QC code with its graph, encoder and transmission layout."""

    def __init__(self, bg: int, Z: int, seed: int | None = None, rows_kept: int = 0,
                 punct_cols: int = 0, n_tx: int | None = None, encoder: bool = True):
        seed = (1 if bg == 1 else 2) if seed is None else seed
        self.bg, self.Z, self.seed = bg, Z, seed
        self.S, self.Kb = base_matrix(bg, Z, seed, rows_kept)
        self.graph = Graph(self.S, Z)
        self.n, self.k = self.graph.n, self.Kb * Z
        self.p0 = punct_cols * Z
        self.n_tx = (self.n - self.p0) if n_tx is None else n_tx
        self.encoder = Encoder(self.S, self.Kb, Z) if encoder else None


def sim(code: Code, *, seed: int, cw0: int, B: int, ebn0_db: float, m: int,
        demap_method: int = DEMAP_MAXLOG, demap_clamp: float = 20.0,
        algo: int = ALGO_MINSUM, schedule: int = SCHED_LAYERED, iters: int = 20, prec: int = 0,
        store: int = STORE_NATIVE, early_stop: bool = False, offset: float = 0.5, clamp: float = 20.0,
        nthreads: int | None = None) -> np.ndarray:
    """Whole chain for codewords [cw0, cw0+B); returns int64
    [info bits, bit errors, blocks, block errors, iterations]."""
    g = code.graph
    counts = np.zeros(5, dtype=np.int64)
    nthreads = nthreads or (os.cpu_count() or 1)
    st = lib().orc_sim(code.encoder._h, g.n, g.m, g.E, g.n_layers, g.n_cls,
                       g.cn_ptr, g.edge_vn, g.edge_cls, g.layer_ptr,
                       code.k, code.p0, code.n_tx, m, demap_method, demap_clamp,
                       algo, schedule, iters, prec, store, int(early_stop), offset, clamp,
                       seed, cw0, B, ebn0_db, counts, nthreads)
    _check(st, "sim")
    return counts
