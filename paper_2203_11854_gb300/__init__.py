"""GB300 QC-LDPC Monte-Carlo hot path: thin Python binding of libldpcx.so.

Every function here has the name of the C entry point it calls (see
``include/ldpcx.h``) and only marshals arguments: torch CUDA tensors supply
device memory and the current stream supplies ``stream``. All computation
runs in the CUDA kernels of ``csrc/``; there is no CPU fallback: when the
library is missing or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import _build

__all__ = [
    "LdpcxError", "Code", "ldpcx_status_str", "ldpcx_sync_status", "qc_ldpc_build", "qc_ldpc_free",
    "qc_ldpc_info", "qc_ldpc_base", "sim_tx", "demap_app", "ldpc_bp_workspace", "ldpc_bp_decode",
    "sim_count", "sim_workspace", "sim_run", "library_path", "load_library", "ldpcx_tune_set", "ldpcx_tune_get",
    "ldpc_bp_decode_noalloc", "ldpc_bp_msg_format", "ldpc_bp_mixed_workspace", "ldpc_bp_decode_mixed", "ldpc_bp_ckpt_bytes", "ldpc_bp_decode_ckpt", "ldpc_bp_backward_workspace",
    "ldpc_bp_backward", "ldpcx_phi", "sim_codewords", "demap_app_prior", "llr_apriori", "llr_mutual_info",
    "ldpc_extrinsic", "DEMAP_OUT_APP", "DEMAP_OUT_EXTRINSIC", "sim_tx_points", "demap_points",
    "demap_points_backward", "map_points_backward", "llr_bce", "PolarCode", "polar_build", "polar_sim_tx",
    "polar_scl_decode", "qc_ldpc_build_base", "qc_alist_parse", "qc_ldpc_alist", "rate_match", "rate_recover",
    "qc_ldpc_shorten", "qam_map_awgn", "ldpcx_fault_set", "FAULT_NONE", "FAULT_ALLOC",
    "LAYERED_MINSUM", "LAYERED_SPA", "FLOOD_MINSUM", "FLOOD_SPA", "MSG_F32", "MSG_F16", "MSG_FIX6",
    "DEMAP_EXACT", "DEMAP_MAXLOG",
]

LAYERED_MINSUM, LAYERED_SPA, FLOOD_MINSUM, FLOOD_SPA = 0, 1, 2, 3
MSG_F32, MSG_F16, MSG_FIX6 = 0, 1, 2
DEMAP_EXACT, DEMAP_MAXLOG = 0, 1
DEMAP_OUT_APP, DEMAP_OUT_EXTRINSIC = 0, 1
FLAG_NONFINITE, FLAG_TIMEOUT = 1, 2
TUNE_L2_PREFETCH, TUNE_ZPT, TUNE_CW_PER_CTA, TUNE_SPECIALISED, TUNE_CN_STATE, TUNE_SCHEDULE = 1, 2, 3, 4, 5, 6
FAULT_NONE, FAULT_ALLOC = 0, 1


class LdpcxError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {ldpcx_status_str(status)} ({status})")


class CodeParams(C.Structure):
    _fields_ = [("bg_shape", C.c_int), ("Z", C.c_int), ("seed", C.c_uint64), ("rows_kept", C.c_int),
                ("punct_cols", C.c_int), ("n_tx", C.c_int)]


class CodeInfo(C.Structure):
    _fields_ = [("Z", C.c_int), ("rows", C.c_int), ("cols", C.c_int), ("kb", C.c_int), ("nnz", C.c_int),
                ("max_row_deg", C.c_int), ("n", C.c_int), ("k", C.c_int), ("n_tx", C.c_int), ("p0", C.c_int),
                ("edges", C.c_int64), ("encodable", C.c_int), ("n_fill", C.c_int)]


class BaseParams(C.Structure):
    _fields_ = [("rows", C.c_int), ("cols", C.c_int), ("kb", C.c_int), ("Z", C.c_int), ("S", C.c_void_p),
                ("punct_cols", C.c_int), ("n_tx", C.c_int)]


class DecodeOpts(C.Structure):
    _fields_ = [("algo", C.c_int), ("iters", C.c_int), ("msg_prec", C.c_int), ("early_stop", C.c_int),
                ("offset", C.c_float), ("clamp", C.c_float), ("weights", C.c_void_p)]


class SimConfig(C.Structure):
    _fields_ = [("code", C.c_void_p), ("m", C.c_int), ("demap_method", C.c_int), ("demap_clamp", C.c_float),
                ("dec", DecodeOpts), ("seed", C.c_uint64), ("cw0", C.c_uint64), ("batch", C.c_int64),
                ("max_batches", C.c_int64), ("min_bit_errors", C.c_int64), ("ebn0_db", C.POINTER(C.c_double)),
                ("n_snr", C.c_int), ("stop_ber", C.c_double), ("use_graph", C.c_int), ("ckpt_path", C.c_char_p),
                ("max_points", C.c_int)]


class BatchGroup(C.Structure):
    _fields_ = [("code", C.c_void_p), ("B", C.c_int64), ("llr_ch", C.c_void_p), ("llr_out", C.c_void_p),
                ("bits_out", C.c_void_p), ("iters_out", C.c_void_p)]


class SimCounts(C.Structure):
    _fields_ = [("bits", C.c_int64), ("bit_errors", C.c_int64), ("blocks", C.c_int64),
                ("block_errors", C.c_int64), ("iter_sum", C.c_int64)]


_lib = None
_lock = threading.Lock()
_vp, _i, _i64, _u64, _f, _sz = C.c_void_p, C.c_int, C.c_int64, C.c_uint64, C.c_float, C.c_size_t

_SIGS = {
    "ldpcx_status_str": ([_i], C.c_char_p),
    "ldpcx_sync_status": ([_vp, C.POINTER(C.c_uint)], _i),
    "qc_ldpc_build": ([C.POINTER(CodeParams), C.POINTER(_vp)], _i),
    "qc_ldpc_free": ([_vp], _i),
    "qc_ldpc_info": ([_vp, C.POINTER(CodeInfo)], _i),
    "qc_ldpc_base": ([_vp, _vp, _i], _i),
    "qc_ldpc_build_base": ([C.POINTER(BaseParams), C.POINTER(_vp)], _i),
    "qc_alist_parse": ([C.c_char_p, _sz, _i, _vp, _i, C.POINTER(_i), C.POINTER(_i)], _i),
    "qc_ldpc_alist": ([_vp, _vp, _sz, C.POINTER(_sz)], _i),
    "qc_ldpc_shorten": ([_vp, _i, C.POINTER(_vp)], _i),
    "qam_map_awgn": ([_vp, _i64, _i, _i, _u64, _u64, _vp, _i64, _vp, _vp], _i),
    "rate_match": ([_vp, _vp, _i64, _i, _i, _i, _i, _vp, _vp], _i),
    "rate_recover": ([_vp, _vp, _i64, _i, _i, _i, _i, _vp, _vp], _i),
    "sim_tx": ([_vp, _u64, _u64, _i64, _i, _vp, _i64, _vp, _vp, _vp], _i),
    "demap_app": ([_vp, _vp, _i64, _i64, _i64, _i, _i, _f, _vp, _vp], _i),
    "sim_codewords": ([_vp, _u64, _u64, _i64, _vp, _vp], _i),
    "demap_app_prior": ([_vp, _vp, _i64, _i64, _i64, _i, _i, _f, _vp, _i, _vp, _vp], _i),
    "llr_apriori": ([_vp, _i64, _i64, _i64, _i64, _f, _u64, _u64, _vp, _vp], _i),
    "llr_mutual_info": ([_vp, _i64, _i64, _vp, _i64, _i64, _vp, _vp], _i),
    "ldpc_extrinsic": ([_vp, _vp, _vp, _i64, _f, _vp, _vp], _i),
    "sim_tx_points": ([_vp, _u64, _u64, _i64, _i, _vp, _vp, _i64, _vp, _vp, _vp], _i),
    "demap_points": ([_vp, _vp, _i64, _i64, _i64, _i, _vp, _i, _f, _vp, _vp], _i),
    "demap_points_backward": ([_vp, _vp, _i64, _i64, _i64, _i, _vp, _f, _vp, _vp, _vp, _vp], _i),
    "map_points_backward": ([_vp, _vp, _i64, _i, _vp, _vp, _vp], _i),
    "llr_bce": ([_vp, _i64, _i64, _vp, _i64, _i64, _f, _vp, _vp, _vp], _i),
    "polar_build": ([_i, _i, _f, _u64, _i, C.POINTER(_vp)], _i),
    "polar_free": ([_vp], _i),
    "polar_info": ([_vp, C.POINTER(_i), C.POINTER(_i), C.POINTER(_i), _vp], _i),
    "polar_sim_tx": ([_vp, _u64, _u64, _i64, _vp, _i64, _vp, _vp, _vp], _i),
    "polar_scl_decode": ([_vp, _vp, _i64, _i, _vp, _vp, _vp], _i),
    "ldpc_bp_workspace": ([_vp, _i64, C.POINTER(DecodeOpts), C.POINTER(_sz)], _i),
    "ldpc_bp_decode": ([_vp, _vp, _i64, C.POINTER(DecodeOpts), _vp, _vp, _vp, _vp, _sz, _vp], _i),
    "ldpc_bp_decode_qam": ([_vp, _vp, _vp, _i64, _i64, _i, _i, _f, C.POINTER(DecodeOpts), _vp, _vp, _vp, _vp, _sz,
                            _vp], _i),
    "sim_count": ([_vp, _vp, _vp, _i64, _i, _vp, _vp], _i),
    "sim_workspace": ([C.POINTER(SimConfig), C.POINTER(_sz)], _i),
    "sim_run": ([C.POINTER(SimConfig), C.POINTER(SimCounts), C.POINTER(_i), _vp, _sz, _vp], _i),
    "ldpc_bp_decode_noalloc": ([_vp, _vp, _i64, C.POINTER(DecodeOpts), _vp, _vp, _vp, _vp], _i),
    "ldpc_bp_msg_format": ([_vp, C.POINTER(DecodeOpts), C.POINTER(_i), C.POINTER(_i64)], _i),
    "ldpcx_phi": ([_vp, _vp, _i64, _i, _vp], _i),
    "ldpc_bp_mixed_workspace": ([C.POINTER(BatchGroup), _i, C.POINTER(DecodeOpts), C.POINTER(_sz)], _i),
    "ldpc_bp_decode_mixed": ([C.POINTER(BatchGroup), _i, C.POINTER(DecodeOpts), _vp, _sz, _vp], _i),
    "ldpc_bp_ckpt_bytes": ([_vp, _i64, C.POINTER(DecodeOpts), C.POINTER(_sz)], _i),
    "ldpc_bp_decode_ckpt": ([_vp, _vp, _i64, C.POINTER(DecodeOpts), _vp, _vp, _vp, _vp, _sz, _vp, _sz, _vp], _i),
    "ldpc_bp_backward_workspace": ([_vp, _i64, C.POINTER(DecodeOpts), C.POINTER(_sz)], _i),
    "ldpc_bp_backward": ([_vp, _vp, _i64, C.POINTER(DecodeOpts), _vp, _sz, _vp, _vp, _vp, _vp, _sz, _vp], _i),
    "ldpcx_tune_set": ([_i, _i], _i),
    "ldpcx_fault_set": ([_i, _i], _i),
    "ldpcx_tune_get": ([_i, C.POINTER(_i)], _i),
}


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = False):
    """Load libldpcx.so (raises when it is missing: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_build.LIB):
                if not build_if_missing:
                    raise ImportError(f"libldpcx.so is not built ({_build.LIB}); run __graft_entry__.build()")
                _build.build()
            L = C.CDLL(_build.LIB)
            for name, (args, res) in _SIGS.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
    return _lib


def _check(st: int, what: str) -> None:
    if st != 0:
        raise LdpcxError(st, what)


def _ptr(t) -> int | None:
    if t is None:
        return None
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    import torch
    return torch.cuda.current_stream().cuda_stream


def _cuda_f32(t, name):
    import torch
    if t.device.type != "cuda" or t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
    return t


def ldpcx_status_str(status: int) -> str:
    return load_library().ldpcx_status_str(status).decode()


def ldpcx_sync_status(stream=None) -> tuple[int, int]:
    """Synchronise and return (status, flags) latched by the kernels since the last call."""
    flags = C.c_uint(0)
    st = load_library().ldpcx_sync_status(_stream(stream), C.byref(flags))
    return st, flags.value


# --------------------------------------------------------------------------- codes
class Code:
    """Owner of an ldpcx_code_t (freed with the object)."""

    def __init__(self, handle: int):
        self.handle = handle
        info = CodeInfo()
        _check(load_library().qc_ldpc_info(handle, C.byref(info)), "qc_ldpc_info")
        self.info = info
        for f, _ in CodeInfo._fields_:
            setattr(self, f, getattr(info, f))

    def base(self):
        import numpy as np
        S = np.zeros(self.rows * self.cols, dtype=np.int16)
        _check(load_library().qc_ldpc_base(self.handle, S.ctypes.data, S.size), "qc_ldpc_base")
        return S.reshape(self.rows, self.cols)

    def close(self):
        if self.handle:
            load_library().qc_ldpc_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def qc_ldpc_build(bg_shape: int, Z: int, seed: int | None = None, rows_kept: int = 0, punct_cols: int = 0,
                  n_tx: int = 0) -> Code:
    seed = (1 if bg_shape == 1 else 2) if seed is None else seed
    p = CodeParams(bg_shape, Z, seed, rows_kept, punct_cols, n_tx)
    h = C.c_void_p()
    _check(load_library().qc_ldpc_build(C.byref(p), C.byref(h)), "qc_ldpc_build")
    return Code(h.value)


def qc_ldpc_build_base(S, Z: int, kb: int, punct_cols: int = 0, n_tx: int = 0) -> Code:
    """Code from a caller-supplied base matrix S ([rows][cols], -1 = zero block, else the shift)."""
    import numpy as np
    S = np.ascontiguousarray(S, dtype=np.int16)
    if S.ndim != 2:
        raise ValueError("S must be a 2-D base matrix")
    p = BaseParams(S.shape[0], S.shape[1], kb, Z, S.ctypes.data, punct_cols, n_tx)
    h = C.c_void_p()
    _check(load_library().qc_ldpc_build_base(C.byref(p), C.byref(h)), "qc_ldpc_build_base")
    return Code(h.value)


def qc_alist_parse(text: str, Z: int):
    """Base matrix ([rows][cols] int16, -1 = zero block) of an alist parity-check matrix of lifting size Z."""
    import numpy as np
    raw = text.encode("ascii")
    rows, cols = _i(), _i()
    lib = load_library()
    _check(lib.qc_alist_parse(raw, len(raw), Z, None, 0, C.byref(rows), C.byref(cols)), "qc_alist_parse")
    S = np.empty((rows.value, cols.value), dtype=np.int16)
    _check(lib.qc_alist_parse(raw, len(raw), Z, S.ctypes.data, S.size, C.byref(rows), C.byref(cols)),
           "qc_alist_parse")
    return S


def qc_ldpc_alist(code: Code) -> str:
    """The code's parity-check matrix as alist text."""
    lib = load_library()
    n = _sz()
    _check(lib.qc_ldpc_alist(code.handle, None, 0, C.byref(n)), "qc_ldpc_alist")
    buf = C.create_string_buffer(n.value + 1)
    _check(lib.qc_ldpc_alist(code.handle, buf, n.value + 1, C.byref(n)), "qc_ldpc_alist")
    return buf.value.decode("ascii")


def qc_ldpc_shorten(code: Code, k: int) -> Code:
    """A new code carrying k information bits: systematic positions k .. kb*Z-1 become filler bits
    (known zeros, not transmitted)."""
    h = C.c_void_p()
    _check(load_library().qc_ldpc_shorten(code.handle, k, C.byref(h)), "qc_ldpc_shorten")
    return Code(h.value)


def rate_match(code: Code, cw, k0: int, ncb: int, E: int, qm: int, out=None, stream=None):
    """Packed transmitted bits [B, ceil(E/32)] (int32) of packed codewords cw [B, ceil(n/32)] (int32, CUDA)."""
    import torch
    B = cw.shape[0]
    if out is None:
        out = torch.empty((B, (E + 31) // 32), dtype=torch.int32, device=cw.device)
    _check(load_library().rate_match(code.handle, _ptr(cw), B, k0, ncb, E, qm, _ptr(out), _stream(stream)),
           "rate_match")
    return out


def rate_recover(code: Code, llr, k0: int, ncb: int, qm: int, out=None, stream=None):
    """Soft buffer [B, ncb] (float32) of received LLRs llr [B, E] (float32, CUDA, transmission order)."""
    import torch
    _cuda_f32(llr, "llr")
    B, E = llr.shape
    if out is None:
        out = torch.empty((B, ncb), dtype=torch.float32, device=llr.device)
    _check(load_library().rate_recover(code.handle, _ptr(llr), B, k0, ncb, E, qm, _ptr(out), _stream(stream)),
           "rate_recover")
    return out


def qc_ldpc_free(code: Code) -> None:
    code.close()


def qc_ldpc_info(code: Code) -> CodeInfo:
    return code.info


def qc_ldpc_base(code: Code):
    return code.base()


# --------------------------------------------------------------------------- transmitter
def sim_tx(code: Code, seed: int, cw0: int, B: int, m: int, no, y_out=None, info_out=None, stream=None):
    """Source + encoder + Gray mapper + AWGN for codewords cw0..cw0+B-1.

    no: CUDA float32 tensor with 1 (shared) or B (per codeword) entries.
    Returns (y [B, S] or [B, S, 2], info [B, ceil(k/32)] int32 view of the packed bits)."""
    import torch
    S = code.n_tx // m
    dev = no.device
    if y_out is None:
        y_out = torch.empty((B, S) if m == 1 else (B, S, 2), dtype=torch.float32, device=dev)
    if info_out is None:
        info_out = torch.empty((B, (code.k + 31) // 32), dtype=torch.int32, device=dev)
    _cuda_f32(no, "no")
    stride = 0 if no.numel() == 1 else 1
    _check(load_library().sim_tx(code.handle, seed, cw0, B, m, _ptr(no), stride, _ptr(y_out), _ptr(info_out),
                                 _stream(stream)), "sim_tx")
    return y_out, info_out


def qam_map_awgn(bits, E: int, m: int, seed: int, cw0: int, no, y_out=None, stream=None):
    """Gray mapper + AWGN on packed bits [B, ceil(E/32)] (int32, CUDA): symbols and noise as sim_tx draws them
    for codewords cw0 .. cw0+B-1. Returns y [B, E] (m = 1) or [B, E/m, 2] float32."""
    import torch
    _cuda_f32(no, "no")
    B = bits.shape[0]
    if y_out is None:
        y_out = torch.empty((B, E) if m == 1 else (B, E // m, 2), dtype=torch.float32, device=bits.device)
    stride = 0 if no.numel() == 1 else 1
    _check(load_library().qam_map_awgn(_ptr(bits), B, E, m, seed, cw0, _ptr(no), stride, _ptr(y_out),
                                       _stream(stream)), "qam_map_awgn")
    return y_out


# --------------------------------------------------------------------------- demapper
def demap_app(y, no, m: int, method: int = DEMAP_EXACT, clamp: float = 20.0, llr_out=None, stream=None):
    """APP demapper: y [B, S] (m = 1) or [B, S, 2] -> LLRs [B, S*m]."""
    import torch
    _cuda_f32(y, "y")
    _cuda_f32(no, "no")
    B, S = y.shape[0], y.shape[1]
    if llr_out is None:
        llr_out = torch.empty((B, S * m), dtype=torch.float32, device=y.device)
    stride = 0 if no.numel() == 1 else 1
    _check(load_library().demap_app(_ptr(y), _ptr(no), stride, B, S, m, method, clamp, _ptr(llr_out),
                                    _stream(stream)), "demap_app")
    return llr_out


def demap_app_prior(y, no, m: int, prior=None, *, method: int = DEMAP_EXACT, clamp: float = 20.0,
                    out_mode: int = DEMAP_OUT_EXTRINSIC, llr_out=None, stream=None):
    """APP demapper with a-priori LLRs prior [B, S*m] (None = zero): a-posteriori (DEMAP_OUT_APP) or
    extrinsic (DEMAP_OUT_EXTRINSIC) LLRs [B, S*m]."""
    import torch
    _cuda_f32(y, "y")
    _cuda_f32(no, "no")
    B, S = y.shape[0], y.shape[1]
    if prior is not None:
        _cuda_f32(prior, "prior")
        assert prior.shape == (B, S * m)
    if llr_out is None:
        llr_out = torch.empty((B, S * m), dtype=torch.float32, device=y.device)
    stride = 0 if no.numel() == 1 else 1
    _check(load_library().demap_app_prior(_ptr(y), _ptr(no), stride, B, S, m, method, clamp,
                                          None if prior is None else _ptr(prior), out_mode, _ptr(llr_out),
                                          _stream(stream)), "demap_app_prior")
    return llr_out


def sim_codewords(code: "Code", seed: int, cw0: int, B: int, out=None, stream=None):
    """The codewords sim_tx sends for (seed, cw0, B), packed: int32 [B, ceil(n/32)]."""
    import torch
    nw = (code.n + 31) // 32
    if out is None:
        out = torch.empty((B, nw), dtype=torch.int32, device="cuda")
    _check(load_library().sim_codewords(code.handle, seed, cw0, B, _ptr(out), _stream(stream)), "sim_codewords")
    return out


def llr_apriori(bits, bit_off: int, N: int, sigma: float, *, seed: int = 0x1DBC, cw0: int = 0, out=None,
                stream=None):
    """Consistent Gaussian a-priori LLRs [B, N] of bits[:, bit_off : bit_off + N] (packed int32 rows)."""
    import torch
    B = bits.shape[0]
    if out is None:
        out = torch.empty((B, N), dtype=torch.float32, device=bits.device)
    _check(load_library().llr_apriori(_ptr(bits), bits.shape[1], bit_off, B, N, sigma, seed, cw0, _ptr(out),
                                      _stream(stream)), "llr_apriori")
    return out


def llr_mutual_info(llr, bits, bit_off: int = 0, acc=None, stream=None):
    """Mutual information between the LLRs [B, N] and bits[:, bit_off : bit_off + N]; returns the float
    (synchronises) unless an accumulator acc (CUDA float64 [2]) is given, which is then updated."""
    import torch
    B, N = llr.shape
    own = acc is None
    if own:
        acc = torch.zeros(2, dtype=torch.float64, device=llr.device)
    _check(load_library().llr_mutual_info(_ptr(llr), B, N, _ptr(bits), bits.shape[1], bit_off, _ptr(acc),
                                          _stream(stream)), "llr_mutual_info")
    if own:
        a = acc.cpu().tolist()
        return 1.0 - a[0] / a[1] if a[1] else float("nan")
    return acc


def ldpc_extrinsic(code: "Code", app, llr_in, *, clamp: float = 20.0, out=None, stream=None):
    """Extrinsic LLRs [B, n_tx] = app[:, p0 : p0 + n_tx] - clip(llr_in), clipped to +-clamp (the decode's clamp)."""
    import torch
    B = llr_in.shape[0]
    if out is None:
        out = torch.empty((B, code.n_tx), dtype=torch.float32, device=llr_in.device)
    _check(load_library().ldpc_extrinsic(code.handle, _ptr(app), _ptr(llr_in), B, clamp, _ptr(out),
                                         _stream(stream)), "ldpc_extrinsic")
    return out


def sim_tx_points(code: "Code", seed: int, cw0: int, B: int, m: int, points, no, y_out=None, cw_out=None,
                  stream=None):
    """sim_tx with the constellation points [2^m, 2] (CUDA float32, point l carries label l, MSB first).
    Returns (y [B, S, 2], packed codewords [B, ceil(n/32)] or None)."""
    import torch
    _cuda_f32(points, "points")
    _cuda_f32(no, "no")
    S = code.n_tx // m
    if y_out is None:
        y_out = torch.empty((B, S, 2), dtype=torch.float32, device=points.device)
    stride = 0 if no.numel() == 1 else 1
    _check(load_library().sim_tx_points(code.handle, seed, cw0, B, m, _ptr(points), _ptr(no), stride, _ptr(y_out),
                                        _ptr(cw_out), _stream(stream)), "sim_tx_points")
    return y_out, cw_out


def demap_points(y, no, m: int, points, *, method: int = DEMAP_EXACT, clamp: float = 20.0, llr_out=None,
                 stream=None):
    """APP demapper over the constellation points [2^m, 2]: y [B, S, 2] -> LLRs [B, S*m]."""
    import torch
    _cuda_f32(y, "y")
    _cuda_f32(no, "no")
    _cuda_f32(points, "points")
    B, S = y.shape[0], y.shape[1]
    if llr_out is None:
        llr_out = torch.empty((B, S * m), dtype=torch.float32, device=y.device)
    stride = 0 if no.numel() == 1 else 1
    _check(load_library().demap_points(_ptr(y), _ptr(no), stride, B, S, m, _ptr(points), method, clamp,
                                       _ptr(llr_out), _stream(stream)), "demap_points")
    return llr_out


def demap_points_backward(y, no, m: int, points, grad_llr, grad_points, *, clamp: float = 20.0, grad_y=None,
                          stream=None):
    """Adjoint of demap_points (exact): returns grad_y [B, S, 2]; adds into grad_points [2^m, 2]."""
    import torch
    B, S = y.shape[0], y.shape[1]
    if grad_y is None:
        grad_y = torch.empty_like(y)
    stride = 0 if no.numel() == 1 else 1
    _check(load_library().demap_points_backward(_ptr(y), _ptr(no), stride, B, S, m, _ptr(points), clamp,
                                                _ptr(grad_llr), _ptr(grad_y), _ptr(grad_points), _stream(stream)),
           "demap_points_backward")
    return grad_y


def map_points_backward(code: "Code", cw, m: int, grad_x, grad_points, stream=None):
    """Adds the symbol gradients grad_x [B, S, 2] into grad_points [2^m, 2] by label."""
    _check(load_library().map_points_backward(code.handle, _ptr(cw), cw.shape[0], m, _ptr(grad_x),
                                              _ptr(grad_points), _stream(stream)), "map_points_backward")
    return grad_points


def llr_bce(llr, bits, bit_off: int = 0, *, scale: float = 1.0, grad=True, stream=None):
    """(sum of ln(1 + exp(-(1-2c) L)) as a CUDA float64 [1] tensor, scale * its gradient [B, N] or None)."""
    import torch
    B, N = llr.shape
    acc = torch.zeros(1, dtype=torch.float64, device=llr.device)
    g = torch.empty_like(llr) if grad else None
    _check(load_library().llr_bce(_ptr(llr), B, N, _ptr(bits), bits.shape[1], bit_off, scale, _ptr(acc), _ptr(g),
                                  _stream(stream)), "llr_bce")
    return acc, g


class PolarCode:
    """Owner of an ldpcx_polar_t: N = 2^n, K information positions (data + CRC)."""

    def __init__(self, handle):
        import numpy as np
        self.handle = handle
        N, K, r = C.c_int(0), C.c_int(0), C.c_int(0)
        _check(load_library().polar_info(handle, C.byref(N), C.byref(K), C.byref(r), None), "polar_info")
        self.N, self.K, self.crc_r = N.value, K.value, r.value
        self.n = self.N.bit_length() - 1
        self.k_data = self.K - self.crc_r
        info = np.zeros(self.K, dtype=np.int32)
        _check(load_library().polar_info(handle, None, None, None, info.ctypes.data), "polar_info")
        self.info = info

    def close(self):
        if self.handle:
            load_library().polar_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def polar_build(n: int, K: int, design_esn0_db: float = 0.0, crc_poly: int = 0, crc_r: int = 0) -> PolarCode:
    h = C.c_void_p()
    _check(load_library().polar_build(n, K, design_esn0_db, crc_poly, crc_r, C.byref(h)), "polar_build")
    return PolarCode(h.value)


def polar_sim_tx(code: PolarCode, seed: int, cw0: int, B: int, no, y_out=None, data_out=None, stream=None):
    """Data bits, CRC, encoder, BPSK and AWGN: (y [B, N], packed data bits [B, ceil(k_data/32)])."""
    import torch
    _cuda_f32(no, "no")
    if y_out is None:
        y_out = torch.empty((B, code.N), dtype=torch.float32, device=no.device)
    if data_out is None:
        data_out = torch.empty((B, (code.k_data + 31) // 32), dtype=torch.int32, device=no.device)
    stride = 0 if no.numel() == 1 else 1
    _check(load_library().polar_sim_tx(code.handle, seed, cw0, B, _ptr(no), stride, _ptr(y_out), _ptr(data_out),
                                       _stream(stream)), "polar_sim_tx")
    return y_out, data_out


def polar_scl_decode(code: PolarCode, llr, L: int = 8, data_out=None, pm_out=None, stream=None):
    """CRC-aided SCL (L = 1: SC) of llr [B, N]: (packed data bits [B, ceil(k_data/32)], path metrics [B])."""
    import torch
    _cuda_f32(llr, "llr")
    B = llr.shape[0]
    if data_out is None:
        data_out = torch.empty((B, (code.k_data + 31) // 32), dtype=torch.int32, device=llr.device)
    if pm_out is None:
        pm_out = torch.empty(B, dtype=torch.float32, device=llr.device)
    _check(load_library().polar_scl_decode(code.handle, _ptr(llr), B, L, _ptr(data_out), _ptr(pm_out),
                                           _stream(stream)), "polar_scl_decode")
    return data_out, pm_out


# --------------------------------------------------------------------------- decoder
def _opts(algo, iters, msg_prec, early_stop, offset, clamp, weights) -> DecodeOpts:
    return DecodeOpts(algo, iters, msg_prec, int(bool(early_stop)), offset, clamp,
                      None if weights is None else weights.data_ptr())


def ldpc_bp_workspace(code: Code, B: int, *, algo: int = LAYERED_MINSUM, iters: int = 20, msg_prec: int = MSG_F32,
                      early_stop: bool = False, offset: float = 0.5, clamp: float = 20.0, weights=None) -> int:
    o = _opts(algo, iters, msg_prec, early_stop, offset, clamp, weights)
    ws = C.c_size_t(0)
    _check(load_library().ldpc_bp_workspace(code.handle, B, C.byref(o), C.byref(ws)), "ldpc_bp_workspace")
    return ws.value


def ldpc_bp_msg_format(code: Code, *, algo: int = LAYERED_MINSUM, iters: int = 20, msg_prec: int = MSG_F32,
                       early_stop: bool = False, offset: float = 0.5, clamp: float = 20.0) -> tuple[bool, int]:
    """(check-node state used?, message-storage bytes per codeword per iteration)."""
    o = _opts(algo, iters, msg_prec, early_stop, offset, clamp, None)
    cs, nb = C.c_int(0), C.c_int64(0)
    _check(load_library().ldpc_bp_msg_format(code.handle, C.byref(o), C.byref(cs), C.byref(nb)),
           "ldpc_bp_msg_format")
    return bool(cs.value), nb.value


def ldpcx_phi(x, *, fast: int = 0, out=None, stream=None):
    """phi(x) = ln(1 + 2/(e^x - 1)) as the decoders evaluate it (x: CUDA float32); fast = 0 library
    functions, 1 (or True) the hardware approximations (the adjoint), 2 the same in bits (the layered and
    flooding check node)."""
    import torch
    assert x.is_cuda and x.dtype == torch.float32 and x.is_contiguous()
    out = torch.empty_like(x) if out is None else out
    _check(load_library().ldpcx_phi(_ptr(x), _ptr(out), x.numel(), int(fast), _stream(stream)), "ldpcx_phi")
    return out


def ldpc_bp_decode(code: Code, llr_ch, *, algo: int = LAYERED_MINSUM, iters: int = 20, msg_prec: int = MSG_F32,
                   early_stop: bool = False, offset: float = 0.5, clamp: float = 20.0, weights=None,
                   llr_out=False, bits_out=True, iters_out=True, ws=None, stream=None):
    """Decode llr_ch [B, n_tx] (CUDA float32).

    llr_out / bits_out / iters_out: a tensor to fill, True to allocate, or
    False/None to skip. ws: a uint8 CUDA tensor of >= ldpc_bp_workspace bytes
    (allocated here when None). Returns (llr_out, bits_out, iters_out)."""
    import torch
    _cuda_f32(llr_ch, "llr_ch")
    B = llr_ch.shape[0]
    dev = llr_ch.device
    if weights is not None:
        _cuda_f32(weights, "weights")
    o = _opts(algo, iters, msg_prec, early_stop, offset, clamp, weights)
    if llr_out is True:
        llr_out = torch.empty((B, code.n), dtype=torch.float32, device=dev)
    if bits_out is True:
        bits_out = torch.empty((B, (code.k + 31) // 32), dtype=torch.int32, device=dev)
    if iters_out is True:
        iters_out = torch.empty((B,), dtype=torch.int32, device=dev)
    llr_out = llr_out if llr_out is not False else None
    bits_out = bits_out if bits_out is not False else None
    iters_out = iters_out if iters_out is not False else None
    need = ldpc_bp_workspace(code, B, algo=algo, iters=iters, msg_prec=msg_prec, early_stop=early_stop,
                             offset=offset, clamp=clamp, weights=weights)
    if ws is None:
        ws = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
    _check(load_library().ldpc_bp_decode(code.handle, _ptr(llr_ch), B, C.byref(o), _ptr(llr_out), _ptr(bits_out),
                                         _ptr(iters_out), _ptr(ws), ws.numel() * ws.element_size(),
                                         _stream(stream)), "ldpc_bp_decode")
    return llr_out, bits_out, iters_out


def ldpc_bp_decode_qam(code: Code, y, no, m: int, *, demap_method: int = DEMAP_EXACT, demap_clamp: float = 20.0,
                       algo: int = LAYERED_MINSUM, iters: int = 20, msg_prec: int = MSG_F32, early_stop: bool = False,
                       offset: float = 0.5, clamp: float = 20.0, llr_out=False, bits_out=True, iters_out=True,
                       ws=None, stream=None):
    """Demapper fused into the layered decoder: received symbols y [B, n_tx/m, 2] ([B, n_tx] for m = 1) and N0
    (one value or [B]) -> the outputs of demap_app followed by ldpc_bp_decode, bit for bit. Outputs and ws as
    ldpc_bp_decode."""
    import torch
    _cuda_f32(y, "y")
    _cuda_f32(no, "no")
    B = y.shape[0]
    dev = y.device
    o = _opts(algo, iters, msg_prec, early_stop, offset, clamp, None)
    if llr_out is True:
        llr_out = torch.empty((B, code.n), dtype=torch.float32, device=dev)
    if bits_out is True:
        bits_out = torch.empty((B, (code.k + 31) // 32), dtype=torch.int32, device=dev)
    if iters_out is True:
        iters_out = torch.empty((B,), dtype=torch.int32, device=dev)
    llr_out = llr_out if llr_out is not False else None
    bits_out = bits_out if bits_out is not False else None
    iters_out = iters_out if iters_out is not False else None
    need = ldpc_bp_workspace(code, B, algo=algo, iters=iters, msg_prec=msg_prec, early_stop=early_stop,
                             offset=offset, clamp=clamp)
    if ws is None:
        ws = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
    stride = 0 if no.numel() == 1 else 1
    _check(load_library().ldpc_bp_decode_qam(code.handle, _ptr(y), _ptr(no), stride, B, m, demap_method,
                                             demap_clamp, C.byref(o), _ptr(llr_out), _ptr(bits_out),
                                             _ptr(iters_out), _ptr(ws), ws.numel() * ws.element_size(),
                                             _stream(stream)), "ldpc_bp_decode_qam")
    return llr_out, bits_out, iters_out


def ldpc_bp_decode_noalloc(code: Code, llr_ch, *, algo: int = LAYERED_MINSUM, iters: int = 20,
                           msg_prec: int = MSG_F32, early_stop: bool = False, offset: float = 0.5,
                           clamp: float = 20.0, weights=None, llr_out=False, bits_out=True, iters_out=True,
                           stream=None):
    """ldpc_bp_decode without a workspace, for callers that cannot allocate device
    memory: the library's fixed scratch array holds the messages, so B is limited
    (see LDPCX_NOALLOC_SCRATCH_BYTES in ldpcx.h). Outputs given as tensors are filled;
    True allocates them here with torch (pass tensors to keep the call allocation-free)."""
    import torch
    _cuda_f32(llr_ch, "llr_ch")
    B = llr_ch.shape[0]
    dev = llr_ch.device
    if weights is not None:
        _cuda_f32(weights, "weights")
    o = _opts(algo, iters, msg_prec, early_stop, offset, clamp, weights)
    if llr_out is True:
        llr_out = torch.empty((B, code.n), dtype=torch.float32, device=dev)
    if bits_out is True:
        bits_out = torch.empty((B, (code.k + 31) // 32), dtype=torch.int32, device=dev)
    if iters_out is True:
        iters_out = torch.empty((B,), dtype=torch.int32, device=dev)
    llr_out = llr_out if llr_out is not False else None
    bits_out = bits_out if bits_out is not False else None
    iters_out = iters_out if iters_out is not False else None
    _check(load_library().ldpc_bp_decode_noalloc(code.handle, _ptr(llr_ch), B, C.byref(o), _ptr(llr_out),
                                                 _ptr(bits_out), _ptr(iters_out), _stream(stream)),
           "ldpc_bp_decode_noalloc")
    return llr_out, bits_out, iters_out


# --------------------------------------------------------------------------- mixed-size batches
def _groups(groups, llr_out):
    import torch
    arr = (BatchGroup * len(groups))()
    outs = []
    for i, (code, llr) in enumerate(groups):
        _cuda_f32(llr, "llr_ch")
        B, dev = llr.shape[0], llr.device
        lo = torch.empty((B, code.n), dtype=torch.float32, device=dev) if llr_out else None
        bits = torch.empty((B, (code.k + 31) // 32), dtype=torch.int32, device=dev)
        its = torch.empty((B,), dtype=torch.int32, device=dev)
        arr[i] = BatchGroup(code.handle, B, llr.data_ptr(), _ptr(lo), bits.data_ptr(), its.data_ptr())
        outs.append((lo, bits, its))
    return arr, outs


def ldpc_bp_mixed_workspace(groups, *, algo: int = LAYERED_MINSUM, iters: int = 20, msg_prec: int = MSG_F16,
                            early_stop: bool = True, offset: float = 0.5, clamp: float = 20.0) -> int:
    arr, _ = _groups(groups, False)
    o = _opts(algo, iters, msg_prec, early_stop, offset, clamp, None)
    n = C.c_size_t(0)
    _check(load_library().ldpc_bp_mixed_workspace(arr, len(groups), C.byref(o), C.byref(n)),
           "ldpc_bp_mixed_workspace")
    return n.value


def ldpc_bp_decode_mixed(groups, *, algo: int = LAYERED_MINSUM, iters: int = 20, msg_prec: int = MSG_F16,
                         early_stop: bool = True, offset: float = 0.5, clamp: float = 20.0, llr_out: bool = False,
                         ws=None, stream=None):
    """Decode a batch mixing codes in one persistent launch.

    groups: list of (Code, llr_ch [B_i, n_tx_i] CUDA float32). Returns a list of
    (llr_out or None, bits [B_i, ceil(k_i/32)], iters [B_i]) per group."""
    import torch
    arr, outs = _groups(groups, llr_out)
    o = _opts(algo, iters, msg_prec, early_stop, offset, clamp, None)
    n = C.c_size_t(0)
    L = load_library()
    _check(L.ldpc_bp_mixed_workspace(arr, len(groups), C.byref(o), C.byref(n)), "ldpc_bp_mixed_workspace")
    if ws is None:
        ws = torch.empty(n.value, dtype=torch.uint8, device=groups[0][1].device)
    _check(L.ldpc_bp_decode_mixed(arr, len(groups), C.byref(o), _ptr(ws), ws.numel(), _stream(stream)),
           "ldpc_bp_decode_mixed")
    return outs


# --------------------------------------------------------------------------- differentiable decoding
def ldpc_bp_ckpt_bytes(code: Code, B: int, *, iters: int = 10, clamp: float = 20.0, weights=None) -> int:
    o = _opts(FLOOD_SPA, iters, MSG_F32, False, 0.0, clamp, weights)
    n = C.c_size_t(0)
    _check(load_library().ldpc_bp_ckpt_bytes(code.handle, B, C.byref(o), C.byref(n)), "ldpc_bp_ckpt_bytes")
    return n.value


def ldpc_bp_decode_ckpt(code: Code, llr_ch, *, iters: int = 10, clamp: float = 20.0, weights=None, ckpt=None,
                        stream=None):
    """Weighted flooding sum-product forward that keeps per-iteration checkpoints.
    Returns (llr_out [B, n], ckpt uint8 tensor)."""
    import torch
    _cuda_f32(llr_ch, "llr_ch")
    B, dev = llr_ch.shape[0], llr_ch.device
    if weights is not None:
        _cuda_f32(weights, "weights")
    o = _opts(FLOOD_SPA, iters, MSG_F32, False, 0.0, clamp, weights)
    need = ldpc_bp_ckpt_bytes(code, B, iters=iters, clamp=clamp, weights=weights)
    if ckpt is None:
        ckpt = torch.empty(need, dtype=torch.uint8, device=dev)
    ws = torch.empty(max(1, ldpc_bp_workspace(code, B, algo=FLOOD_SPA, iters=iters, clamp=clamp, weights=weights)),
                     dtype=torch.uint8, device=dev)
    llr_out = torch.empty((B, code.n), dtype=torch.float32, device=dev)
    _check(load_library().ldpc_bp_decode_ckpt(code.handle, _ptr(llr_ch), B, C.byref(o), _ptr(llr_out), None, None,
                                              _ptr(ws), ws.numel(), _ptr(ckpt), ckpt.numel(), _stream(stream)),
           "ldpc_bp_decode_ckpt")
    return llr_out, ckpt


def ldpc_bp_backward_workspace(code: Code, B: int, *, iters: int = 10, clamp: float = 20.0, weights=None) -> int:
    o = _opts(FLOOD_SPA, iters, MSG_F32, False, 0.0, clamp, weights)
    n = C.c_size_t(0)
    _check(load_library().ldpc_bp_backward_workspace(code.handle, B, C.byref(o), C.byref(n)),
           "ldpc_bp_backward_workspace")
    return n.value


def ldpc_bp_backward(code: Code, llr_ch, ckpt, grad_llr_out, *, iters: int = 10, clamp: float = 20.0, weights=None,
                     grad_weights=None, stream=None):
    """Adjoint of ldpc_bp_decode_ckpt. Returns (grad_llr_ch [B, n_tx], grad_weights [iters, nnz] or None);
    grad_weights, when given, is accumulated into."""
    import torch
    _cuda_f32(llr_ch, "llr_ch")
    _cuda_f32(grad_llr_out, "grad_llr_out")
    B, dev = llr_ch.shape[0], llr_ch.device
    if weights is not None:
        _cuda_f32(weights, "weights")
        if grad_weights is None:
            grad_weights = torch.zeros_like(weights)
    o = _opts(FLOOD_SPA, iters, MSG_F32, False, 0.0, clamp, weights)
    ws = torch.empty(max(1, ldpc_bp_backward_workspace(code, B, iters=iters, clamp=clamp, weights=weights)),
                     dtype=torch.uint8, device=dev)
    grad_llr = torch.empty_like(llr_ch)
    _check(load_library().ldpc_bp_backward(code.handle, _ptr(llr_ch), B, C.byref(o), _ptr(ckpt), ckpt.numel(),
                                           _ptr(grad_llr_out), _ptr(grad_llr), _ptr(grad_weights), _ptr(ws),
                                           ws.numel(), _stream(stream)), "ldpc_bp_backward")
    return grad_llr, grad_weights


# --------------------------------------------------------------------------- counting and sweeps
def sim_count(ref, hat, iters, k: int, counts, stream=None):
    """Accumulate {bits, bit errors, blocks, block errors, iterations} into counts (CUDA int64[5])."""
    B = ref.shape[0]
    _check(load_library().sim_count(_ptr(ref), _ptr(hat), _ptr(iters), B, k, _ptr(counts), _stream(stream)),
           "sim_count")
    return counts


def _sim_config(code: Code, ebn0_db, *, m, demap_method, demap_clamp, algo, iters, msg_prec, early_stop, offset,
                clamp, seed, cw0, batch, max_batches, min_bit_errors, stop_ber, use_graph, ckpt_path, max_points):
    eb = (C.c_double * len(ebn0_db))(*ebn0_db)
    path = None if ckpt_path is None else os.fsencode(ckpt_path)
    cfg = SimConfig(code.handle, m, demap_method, demap_clamp,
                    _opts(algo, iters, msg_prec, early_stop, offset, clamp, None), seed, cw0, batch, max_batches,
                    min_bit_errors, C.cast(eb, C.POINTER(C.c_double)), len(ebn0_db), stop_ber, int(bool(use_graph)),
                    path, max_points)
    return cfg, (eb, path)


_SIM_DEFAULTS = dict(m=4, demap_method=DEMAP_MAXLOG, demap_clamp=20.0, algo=LAYERED_MINSUM, iters=20,
                     msg_prec=MSG_F16, early_stop=False, offset=0.5, clamp=20.0, seed=0x1DBC, cw0=0, batch=1024,
                     max_batches=1, min_bit_errors=0, stop_ber=0.0, use_graph=True, ckpt_path=None, max_points=0)


def sim_workspace(code: Code, ebn0_db, **kw) -> int:
    cfg, _keep = _sim_config(code, ebn0_db, **{**_SIM_DEFAULTS, **kw})
    ws = C.c_size_t(0)
    _check(load_library().sim_workspace(C.byref(cfg), C.byref(ws)), "sim_workspace")
    return ws.value


def sim_run(code: Code, ebn0_db, ws=None, stream=None, device=None, **kw):
    """Monte-Carlo sweep; returns a list of dicts (one per point run, restored points of a checkpoint included).
    ckpt_path: the sweep's checkpoint file (written after every point, resumed from when present);
    max_points: points to run in this call (0 = all)."""
    import torch
    args = {**_SIM_DEFAULTS, **kw}
    cfg, _keep = _sim_config(code, list(ebn0_db), **args)
    need = C.c_size_t(0)
    _check(load_library().sim_workspace(C.byref(cfg), C.byref(need)), "sim_workspace")
    if ws is None:
        ws = torch.empty(need.value, dtype=torch.uint8, device=device or "cuda")
    out = (SimCounts * max(1, len(ebn0_db)))()
    pts = C.c_int(0)
    _check(load_library().sim_run(C.byref(cfg), out, C.byref(pts), _ptr(ws), ws.numel(), _stream(stream)),
           "sim_run")
    return [dict(ebn0_db=float(ebn0_db[i]), bits=out[i].bits, bit_errors=out[i].bit_errors, blocks=out[i].blocks,
                 block_errors=out[i].block_errors, iter_sum=out[i].iter_sum) for i in range(pts.value)]


def ldpcx_tune_set(key: int, value: int) -> None:
    _check(load_library().ldpcx_tune_set(key, value), "ldpcx_tune_set")


def ldpcx_fault_set(kind: int, after: int = 0) -> None:
    """Arm (FAULT_ALLOC: the allocation after `after` more fails once with LDPCX_E_NOMEM) or disarm (FAULT_NONE)
    the library's host-side fault injector."""
    _check(load_library().ldpcx_fault_set(kind, after), "ldpcx_fault_set")


def ldpcx_tune_get(key: int) -> int:
    v = C.c_int(0)
    _check(load_library().ldpcx_tune_get(key, C.byref(v)), "ldpcx_tune_get")
    return v.value
