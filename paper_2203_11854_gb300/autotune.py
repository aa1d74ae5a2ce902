"""Autotuner for the decoder's launch knobs (ldpcx_tune_set).

For a (code, algorithm, message format, iterations, early stop) on the current
device it times every candidate setting of the knobs with CUDA events on a
batch of random LLRs, checks that every candidate gives the same outputs bit
for bit as the first one (knobs must not change results), and keeps the
fastest. Results are cached in a JSON file keyed by the device name and the
decode shape; apply() sets the cached knobs before decoding.

Knobs: LDPCX_TUNE_CW_PER_CTA (codewords per CTA) everywhere; with per-edge
messages LDPCX_TUNE_L2_PREFETCH (message-span prefetch distance of the layered
kernels); with check-node state LDPCX_TUNE_ZPT (one or two check nodes per
thread). Layer order is not a knob: changing it changes the decoder's results.
"""
from __future__ import annotations

import json
import os

import torch

from . import (TUNE_CW_PER_CTA, TUNE_L2_PREFETCH, TUNE_ZPT, ldpc_bp_decode, ldpc_bp_msg_format,
               ldpc_bp_workspace, ldpcx_tune_get, ldpcx_tune_set)

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "ldpcx", "autotune.json")


def _key(code, algo, msg_prec, iters, early_stop):
    dev = torch.cuda.get_device_name()
    return f"{dev}|Z{code.Z}|{code.rows}x{code.cols}|nnz{code.nnz}|algo{algo}|msg{msg_prec}|it{iters}|es{int(early_stop)}"


def _candidates(code, algo=0, msg_prec=1, iters=20):
    auto_g = max(1, 384 // code.Z)
    gs = sorted({0} | {g for g in (auto_g // 2, auto_g // 4) if g >= 1})
    cn_state, _ = ldpc_bp_msg_format(code, algo=algo, iters=iters, msg_prec=msg_prec)
    if cn_state:
        zpts = (0, 2) if code.Z % 2 == 0 else (0,)
        return [{"l2_prefetch": 0, "cw_per_cta": g, "zpt": z} for z in zpts for g in gs]
    return [{"l2_prefetch": pf, "cw_per_cta": g, "zpt": 0} for pf in (0, 1, 2, 4) for g in gs]


def _set(knobs):
    ldpcx_tune_set(TUNE_L2_PREFETCH, knobs["l2_prefetch"])
    ldpcx_tune_set(TUNE_CW_PER_CTA, knobs["cw_per_cta"])
    ldpcx_tune_set(TUNE_ZPT, knobs.get("zpt", 0))


def load_cache(path=None) -> dict:
    path = path or os.environ.get("LDPCX_AUTOTUNE_CACHE", DEFAULT_CACHE)
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path=None) -> None:
    path = path or os.environ.get("LDPCX_AUTOTUNE_CACHE", DEFAULT_CACHE)
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(code, *, B: int = 1024, algo: int = 0, msg_prec: int = 1, iters: int = 20, early_stop: bool = False,
         reps: int = 3, cache_path=None, candidates=None, seed: int = 0) -> dict:
    """Time the candidates, return {"best": knobs, "timings": [...]} and store best in the cache."""
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    llr = (2.0 + 2.0 * torch.randn((B, code.n_tx), device="cuda", generator=gen)).float()
    dec = dict(algo=algo, iters=iters, msg_prec=msg_prec, early_stop=early_stop)
    ws = torch.empty(max(1, ldpc_bp_workspace(code, B, **dec)), dtype=torch.uint8, device="cuda")
    saved = {"l2_prefetch": ldpcx_tune_get(TUNE_L2_PREFETCH), "cw_per_cta": ldpcx_tune_get(TUNE_CW_PER_CTA),
             "zpt": ldpcx_tune_get(TUNE_ZPT)}
    timings, ref = [], None
    try:
        for knobs in (candidates or _candidates(code, algo, msg_prec, iters)):
            _set(knobs)
            out = ldpc_bp_decode(code, llr, **dec, llr_out=True, ws=ws)
            if ref is None:
                ref = out
            elif not all(torch.equal(a, b) for a, b in zip(out, ref)):
                raise RuntimeError(f"tuning knobs {knobs} changed the decoder's results")
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(reps):
                ldpc_bp_decode(code, llr, **dec, bits_out=False, iters_out=False, ws=ws)
            b.record()
            torch.cuda.synchronize()
            timings.append({**knobs, "ms": a.elapsed_time(b) / reps})
    finally:
        _set(saved)
    best = min(timings, key=lambda t: t["ms"])
    best = {"l2_prefetch": best["l2_prefetch"], "cw_per_cta": best["cw_per_cta"], "zpt": best.get("zpt", 0),
            "ms": best["ms"], "B": B}
    cache = load_cache(cache_path)
    cache[_key(code, algo, msg_prec, iters, early_stop)] = best
    save_cache(cache, cache_path)
    return {"best": best, "timings": timings}


def apply(code, *, algo: int = 0, msg_prec: int = 1, iters: int = 20, early_stop: bool = False, cache_path=None):
    """Set the cached knobs for this decode shape (automatic settings when none are cached)."""
    best = load_cache(cache_path).get(_key(code, algo, msg_prec, iters, early_stop))
    _set(best or {"l2_prefetch": 0, "cw_per_cta": 0, "zpt": 0})
    return best
