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
tune_mixed() tunes the persistent mixed-code launch on the caller's batch (the
cap on the codewords of one work item), keyed by the batch's code mix.
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


def _mixed_key(groups, algo, msg_prec, iters, early_stop):
    """The batch's code mix: per group its shape and codeword count, in group order."""
    dev = torch.cuda.get_device_name()
    mix = ";".join(f"Z{c.Z}r{c.rows}c{c.cols}n{c.n_tx}f{c.n_fill}B{int(l.shape[0])}" for c, l in groups)
    return f"{dev}|mixed|{mix}|algo{algo}|msg{msg_prec}|it{iters}|es{int(early_stop)}"


def tune_mixed(groups, *, algo: int = 0, msg_prec: int = 1, iters: int = 20, early_stop: bool = True, reps: int = 3,
               cache_path=None, candidates=(0, 12, 8, 6, 4, 2)) -> dict:
    """Tune the persistent mixed-code launch (ldpc_bp_decode_mixed) on the caller's own batch: the cap on the
    codewords of one work item (LDPCX_TUNE_CW_PER_CTA). Every candidate must give the same outputs bit for bit;
    the fastest is cached under the batch's code mix."""
    from . import ldpc_bp_decode_mixed, ldpc_bp_mixed_workspace
    dec = dict(algo=algo, iters=iters, msg_prec=msg_prec, early_stop=early_stop)
    saved = ldpcx_tune_get(TUNE_CW_PER_CTA)
    timings, ref = [], None
    try:
        for g in candidates:
            ldpcx_tune_set(TUNE_CW_PER_CTA, g)
            ws = torch.empty(ldpc_bp_mixed_workspace(groups, **dec), dtype=torch.uint8, device="cuda")
            out = ldpc_bp_decode_mixed(groups, **dec, llr_out=True, ws=ws)
            flat = [t for o in out for t in o if t is not None]
            if ref is None:
                ref = flat
            elif not all(torch.equal(a, b) for a, b in zip(flat, ref)):
                raise RuntimeError(f"codewords per item {g} changed the decoder's results")
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(reps):
                ldpc_bp_decode_mixed(groups, **dec, ws=ws)
            b.record()
            torch.cuda.synchronize()
            timings.append({"cw_per_cta": g, "ms": a.elapsed_time(b) / reps})
            del ws
    finally:
        ldpcx_tune_set(TUNE_CW_PER_CTA, saved)
    best = dict(min(timings, key=lambda t: t["ms"]))
    cache = load_cache(cache_path)
    cache[_mixed_key(groups, algo, msg_prec, iters, early_stop)] = best
    save_cache(cache, cache_path)
    return {"best": best, "timings": timings}


def apply_mixed(groups, *, algo: int = 0, msg_prec: int = 1, iters: int = 20, early_stop: bool = True,
                cache_path=None):
    """Set the cached work-item cap for this code mix (automatic when none is cached)."""
    best = load_cache(cache_path).get(_mixed_key(groups, algo, msg_prec, iters, early_stop))
    ldpcx_tune_set(TUNE_CW_PER_CTA, best["cw_per_cta"] if best else 0)
    return best


def apply(code, *, algo: int = 0, msg_prec: int = 1, iters: int = 20, early_stop: bool = False, cache_path=None):
    """Set the cached knobs for this decode shape (automatic settings when none are cached)."""
    best = load_cache(cache_path).get(_key(code, algo, msg_prec, iters, early_stop))
    _set(best or {"l2_prefetch": 0, "cw_per_cta": 0, "zpt": 0})
    return best
