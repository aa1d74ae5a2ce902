#!/usr/bin/env python3
"""Throughput of the QC-LDPC Monte-Carlo hot path on GB300.

Workload (BG1-shaped Z=384 full-size case): seeded BG1-shaped 46x68 base
matrix, Z = 384 (n = 26112, k = 8448, the first 2Z systematic bits
punctured, n_tx = 25344), 16-QAM Gray, AWGN at Eb/N0 = 2.0 dB, batch of 4096
codewords, layered offset min-sum (beta 0.5), 20 iterations without early
stop, FP16 messages with FP32 arithmetic.

One step = one Monte-Carlo batch through the whole device path: Philox
source + dual-diagonal encoder + Gray mapper + AWGN (sim_tx) -> APP demapper
fused into the layered BP decoder's channel load (ldpc_bp_decode_qam; with
--unfused, demap_app then ldpc_bp_decode) -> error count (sim_count). Metric: decoded information Gbit/s = ranks x B x k / step time;
edge-updates/s = ranks x B x E x iterations / step time.

Timing: W warm-up steps, then K timed steps between barriers and device
synchronisations, CUDA events on the launching stream, max over ranks.
Every buffer (y 208 MB, messages 893 MB; LLRs 406 MB with --unfused) is
larger than L2, so no flush is needed.

--impl reference times the CPU oracle (the reference arm of this repository:
the paper ships no code) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import datetime
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "decoded info Gbit/s & edge-updates/s, 1 GB300, BG1 Z=384 20-iter; FP16 vs FP32 @ BER 1e-4"
BG, Z, PUNCT, B, M, EBN0, ITERS, OFFSET, CLAMP = 1, 384, 2, 4096, 4, 2.0, 20, 0.5, 20.0
SEED = 0x1DBC | (2 << 32)
PROFILE = os.path.join(ROOT, "profiles", "decode_layered_minsum_f16_bg1_z384.md")


def workload_config(batch=None):
    batch = B if batch is None else batch
    return {"workload": "BG1-shaped 46x68 seeded QC-LDPC (seed 1), Z=384, batch %d, 16-QAM, AWGN Eb/N0 %.1f dB, "
                        "layered offset min-sum (0.5), 20 iterations, FP16 messages" % (batch, EBN0),
            "code": "BG1-shaped 46x68, 316 blocks, Z=384, n=26112, k=8448, 2Z punctured",
            "batch": batch, "modulation": "16-QAM", "ebn0_db": EBN0, "iters": ITERS, "msg": "fp16",
            "l2": "inputs larger than L2 (y %d MB, LLR %d MB, message workspace %d MB): no flush"
                  % (batch * 6336 * 8 >> 20, batch * 25344 * 4 >> 20, batch * 121344 * 2 >> 20)}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class Clocks:
    """Samples nvidia-smi SM clocks and throttle reasons every 20 ms; keeps the samples whose
    timestamps fall inside the timed region (begin() / end() mark it on the host clock)."""

    Q = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.proc, self.path = index, None, None
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.path = f"/tmp/ldpcx_clocks_{os.getpid()}.csv"
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            t = time.time()
            while time.time() - t < 5.0 and os.path.getsize(self.path) == 0:
                time.sleep(0.01)  # sampling has started before the timed region does
        except Exception:
            self.proc = None

    def begin(self):
        self.t0 = time.time()

    def end(self):
        self.t1 = time.time()

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) != 8:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                continue
            rows.append((ts, parts[1:]))
        os.remove(self.path)
        inside = [r for ts, r in rows if self.t0 is not None and self.t0 <= ts <= self.t1]
        if not inside:  # a region shorter than the sampling period: the samples nearest to it
            mid = 0.5 * (self.t0 + self.t1) if self.t0 is not None else 0.0
            inside = [r for ts, r in sorted(rows, key=lambda x: abs(x[0] - mid))[:2]]
        if not inside:
            return None
        sm = [float(r[0]) for r in inside if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in inside if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in inside for i in range(4) if r[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(inside), "interval_ms": 20}


KERNEL_SOURCES = ("decode_kernels.cuh", "demap.cuh", "decode_cns.cuh", "decode_cns_sched.cuh",
                  "decode_cns_sched_f16.cu")  # profiled kernel


def decoder_digest():
    """sha256[:16] over the profiled kernel's sources, to tell whether an ncu summary is current."""
    src = os.path.join(ROOT, "paper_2203_11854_gb300", "csrc")
    blob = b"".join(open(os.path.join(src, f), "rb").read() for f in KERNEL_SOURCES)
    return hashlib.sha256(blob).hexdigest()[:16]


def profile_traffic():
    """dram bytes per codeword from the committed ncu summary, if the decoder sources are unchanged since."""
    try:
        text = open(PROFILE).read()
    except OSError:
        return None, None
    vals = {}
    for line in text.splitlines():
        if ": " in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(": ", 1)
            vals[k.strip()] = v.strip().strip("`")
    digest = decoder_digest()
    if vals.get("kernel sources sha256[:16]") != digest:
        return None, vals.get("kernel sources sha256[:16]")
    try:
        return float(vals["dram bytes per codeword (full-launch scale)"]), digest
    except (KeyError, ValueError):
        return None, digest


def profile_sections(name):
    """Per-kernel figures of a committed ncu summary under profiles/: a list of dicts (one per "### " section, or
    the whole file), each with "current" = True when the sources it names hash as they did at capture time."""
    try:
        text = open(os.path.join(ROOT, "profiles", name)).read()
    except OSError:
        return []
    secs, cur = [], {}
    for line in text.splitlines():
        if line.startswith("### "):
            if cur:
                secs.append(cur)
            cur = {"kernel": line[4:].strip().strip("`")}
        elif ": " in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(": ", 1)
            cur[k.strip()] = v.strip().strip("`")
    if cur:
        secs.append(cur)
    src = os.path.join(ROOT, "paper_2203_11854_gb300", "csrc")
    for sec in secs:
        files = sec.get("kernel sources hashed", "").split(" (")[0].split(" + ")
        try:
            blob = b"".join(open(os.path.join(src, f.strip()), "rb").read() for f in files if f.strip())
            sec["current"] = bool(blob) and hashlib.sha256(blob).hexdigest()[:16] == sec.get("kernel sources sha256[:16]")
        except OSError:
            sec["current"] = False
    return secs


def issue_peak():
    """Warp instructions per second the GPU can issue: SMs x 4 schedulers x the maximum SM clock."""
    import torch
    pk, _ = peaks()
    return torch.cuda.get_device_properties(0).multi_processor_count * 4 * pk.get("sm_max_mhz", 2070.0) * 1e6


def inst_per_32_edges(profile, kernel_sub=None, key="warp instructions per 32 edge updates"):
    """Warp instructions per 32 edge updates (the figure named key) from a current ncu summary, or None."""
    for sec in profile_sections(profile):
        if kernel_sub and kernel_sub not in sec.get("kernel", ""):
            continue
        if sec.get("current") and key in sec:
            return float(sec[key])
    return None


def host_cpu():
    """Architecture and, where the kernel reports one, the model name of the host CPU."""
    import platform
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return f"{platform.machine()}" + (f", {model}" if model else "")


def cpu_baseline(seconds=12.0, ebn0=EBN0):
    """The oracle as it stands (FP64, layered min-sum with the FP16 message store), whole chain, on all
    host cores, for a bounded sample of codewords of the same workload."""
    import oracle
    code = oracle.Code(BG, Z, punct_cols=PUNCT)
    cores = os.cpu_count() or 1
    done, t_total, cw0 = 0, 0.0, 1 << 40
    chunk = max(cores, 8)
    while t_total < seconds and done < 20000:
        t0 = time.perf_counter()
        oracle.sim(code, seed=SEED, cw0=cw0 + done, B=chunk, ebn0_db=ebn0, m=M, demap_method=oracle.DEMAP_MAXLOG,
                   algo=oracle.ALGO_MINSUM, iters=ITERS, prec=0, store=oracle.STORE_F16, offset=OFFSET,
                   clamp=CLAMP, nthreads=cores)
        t_total += time.perf_counter() - t0
        done += chunk
    k = code.k
    # the same chain on one core, a shorter sample
    t1, done1 = 0.0, 0
    while t1 < seconds / 4 and done1 < 2000:
        t0 = time.perf_counter()
        oracle.sim(code, seed=SEED, cw0=cw0 + done + done1, B=2, ebn0_db=ebn0, m=M,
                   demap_method=oracle.DEMAP_MAXLOG, algo=oracle.ALGO_MINSUM, iters=ITERS, prec=0,
                   store=oracle.STORE_F16, offset=OFFSET, clamp=CLAMP, nthreads=1)
        t1 += time.perf_counter() - t0
        done1 += 2
    return {"value": done * k / t_total / 1e9, "unit": "Gbit/s", "cores": cores, "kind": "oracle",
            "cpu": host_cpu(),
            "one_core": {"value": done1 * k / t1 / 1e9, "unit": "Gbit/s", "codewords": done1,
                         "seconds": round(t1, 2)},
            "sample": f"{done} codewords of the workload (FP64 oracle chain: source, GF(2) encoder, mapper, AWGN, "
                      f"max-log demapper, layered min-sum with FP16 message store, 20 iterations), {t_total:.1f} s",
            "codewords_per_s": done / t_total}


def dist_setup(n_gpus):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world != n_gpus and world > 1:
        raise SystemExit(f"--gpus {n_gpus} but WORLD_SIZE {world}")
    return rank, world, local


def run_reference(args):
    rank, world, local = dist_setup(args.gpus)
    if rank != 0:
        return
    import oracle
    code = oracle.Code(BG, Z, punct_cols=PUNCT)
    cores = os.cpu_count() or 1
    per_step = max(cores, 8)
    for i in range(args.warmup):
        oracle.sim(code, seed=SEED, cw0=i * per_step, B=per_step, ebn0_db=EBN0, m=M,
                   demap_method=oracle.DEMAP_MAXLOG, iters=ITERS, store=oracle.STORE_F16, nthreads=cores)
    times = []
    for i in range(args.steps):
        t0 = time.perf_counter()
        oracle.sim(code, seed=SEED, cw0=(args.warmup + i) * per_step, B=per_step, ebn0_db=EBN0, m=M,
                   demap_method=oracle.DEMAP_MAXLOG, iters=ITERS, store=oracle.STORE_F16, nthreads=cores)
        times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    value = per_step * code.k / t / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Gbit/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(),
            "cpu_baseline": {"value": value, "unit": "Gbit/s", "cores": cores, "kind": "oracle", "cpu": host_cpu(),
                             "sample": f"{per_step} codewords per step of the workload through the FP64 oracle chain"},
            "e2e": {"value": value, "unit": "Gbit/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_gpu(args):
    import torch
    rank, world, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2203_11854_gb300 as lx
    lx.load_library()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    code = lx.qc_ldpc_build(BG, Z, punct_cols=PUNCT)
    S = code.n_tx // M
    kw = (code.k + 31) // 32
    r = code.k / code.n_tx
    n0 = torch.tensor([1.0 / (r * M * 10 ** (EBN0 / 10))], dtype=torch.float32, device=dev)
    # two buffer sets: step i + 1's transmitter and demapper run on their own stream while step i decodes
    fused = not args.unfused
    bufs = [dict(y=torch.empty((B, S, 2), dtype=torch.float32, device=dev),
                 info=torch.empty((B, kw), dtype=torch.int32, device=dev),
                 llr=None if fused else torch.empty((B, code.n_tx), dtype=torch.float32, device=dev),
                 bits=torch.empty((B, kw), dtype=torch.int32, device=dev),
                 its=torch.empty((B,), dtype=torch.int32, device=dev)) for _ in range(2)]
    y, info, llr, bits, its = (bufs[0][key] for key in ("y", "info", "llr", "bits", "its"))
    counts = torch.zeros(5, dtype=torch.int64, device=dev)
    dec = dict(algo=lx.LAYERED_MINSUM, iters=ITERS, msg_prec=lx.MSG_F16, offset=OFFSET, clamp=CLAMP)
    ws = torch.empty(lx.ldpc_bp_workspace(code, B, **dec), dtype=torch.uint8, device=dev)
    from paper_2203_11854_gb300 import multi
    cw_base = multi.rank_cw_base(rank)  # disjoint codeword (Philox counter) ranges per rank

    # The decoder's stream has the higher priority, so its CTAs are dispatched first and the transmitter (and,
    # unfused, the demapper) of the next step only take the SM slots that the decoder's last, partial wave leaves
    # idle (4096 codewords on 2 x 152 slots: 13.5 waves). Every step still runs all of its kernels.
    dec_stream = torch.cuda.Stream(device=dev, priority=-1)
    tx_stream = torch.cuda.Stream(device=dev, priority=0)
    ev_rx = [torch.cuda.Event() for _ in range(2)]    # demapper output of buffer j is ready
    ev_free = [torch.cuda.Event() for _ in range(2)]  # the error count has consumed buffer j

    def step(i, timed_decode=None):
        b = bufs[i & 1]
        tx_stream.wait_event(ev_free[i & 1])
        lx.sim_tx(code, SEED, cw_base + i * B, B, M, n0, y_out=b["y"], info_out=b["info"], stream=tx_stream)
        if not fused:
            lx.demap_app(b["y"], n0, M, method=lx.DEMAP_MAXLOG, clamp=CLAMP, llr_out=b["llr"], stream=tx_stream)
        ev_rx[i & 1].record(tx_stream)
        dec_stream.wait_event(ev_rx[i & 1])
        if timed_decode is not None:
            timed_decode[0].record(dec_stream)
        if fused:
            lx.ldpc_bp_decode_qam(code, b["y"], n0, M, demap_method=lx.DEMAP_MAXLOG, demap_clamp=CLAMP, **dec,
                                  llr_out=False, bits_out=b["bits"], iters_out=b["its"], ws=ws, stream=dec_stream)
        else:
            lx.ldpc_bp_decode(code, b["llr"], **dec, llr_out=False, bits_out=b["bits"], iters_out=b["its"], ws=ws,
                              stream=dec_stream)
        if timed_decode is not None:
            timed_decode[1].record(dec_stream)
        lx.sim_count(b["info"], b["bits"], b["its"], code.k, counts, stream=dec_stream)
        ev_free[i & 1].record(dec_stream)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    st, flags = lx.ldpcx_sync_status()
    if st != 0:
        raise SystemExit(f"device status after warm-up: {lx.ldpcx_status_str(st)}")
    counts.zero_()

    clocks = Clocks(local)
    dec_ms = []
    dec_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.begin()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(dec_stream)
    tx_stream.wait_event(t_start)  # no transmitter work of a timed step starts before the timed region
    for i in range(args.steps):
        step(args.warmup + i, dec_ev[i])
    t_end.record(dec_stream)  # the last count follows every kernel of every step on both streams
    torch.cuda.synchronize()
    clocks.end()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    elapsed_ms = t_start.elapsed_time(t_end)
    dec_ms = [a.elapsed_time(b) for a, b in dec_ev]
    elapsed_ms = multi.max_time(elapsed_ms, device=dev)
    c = counts.cpu().tolist()
    ms_per_step = elapsed_ms / args.steps
    value = world * B * code.k / (ms_per_step * 1e-3) / 1e9
    edge_updates = world * B * code.edges * ITERS / (ms_per_step * 1e-3)

    # decode-kernel roofline: algorithmic bytes per launch / mean decode launch time. The message
    # bytes are those of the storage format the decoder uses (check-node state for layered min-sum):
    # one read and one write per iteration except the first read and the last write; the channel input is
    # the received symbols (8 B each) with the demapper fused, else the LLRs (4 B each).
    cn_state, msg_cw = lx.ldpc_bp_msg_format(code, **{k: dec[k] for k in ("algo", "iters", "msg_prec")})
    alg_bytes = B * (msg_cw * 2 * (ITERS - 1) + (8 * S if fused else 4 * code.n_tx) + code.k / 8)
    dec_mean = sum(dec_ms) / len(dec_ms)
    pk, pk_kind = peaks()
    achieved = alg_bytes / (dec_mean * 1e-3) / 1e9
    traffic_cw, _ = profile_traffic()
    ipe = inst_per_32_edges("decode_layered_minsum_f16_bg1_z384.md") if cn_state else None
    issue_frac = None if ipe is None else ipe * B * code.edges * ITERS / (dec_mean * 1e-3) / 32 / issue_peak()

    result = None
    if rank == 0:
        variants = {}
        if not args.quick:
            if llr is None:  # the variants decode LLRs: demap the last buffer's symbols once
                llr = lx.demap_app(y, n0, M, method=lx.DEMAP_MAXLOG, clamp=CLAMP)
            variants = measure_variants(lx, code, llr, bits, its, stream, args, pk)
            variants["mixed_batch"] = measure_mixed(lx, stream, args, pk)
            variants["sweep_256qam"] = measure_sweep(lx, code, pk)
            variants["grad_step"] = measure_grad_step(lx)
            variants["flood_spa_z8"] = measure_flood_z8(lx)
            variants["polar_scl"] = measure_polar(lx)
        e2e = measure_e2e(lx, code, y, info, n0, dec, stream, args, dev, fused=fused)
        cpu = None if (world > 1 or args.no_cpu) else cpu_baseline(args.cpu_seconds)
        result = {
            "metric": METRIC, "value": value, "unit": "Gbit/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "msg_dtype": "f16", "data": "synthetic",
            "config": workload_config(),
            "edge_updates_per_s": edge_updates,
            "codewords_per_s": world * B / (ms_per_step * 1e-3),
            "ber": c[1] / c[0] if c[0] else None, "bler": c[3] / c[2] if c[2] else None,
            "decode_ms_per_launch": dec_mean,
            "decode_ms_median": statistics.median(dec_ms),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                         "frac": achieved / pk["hbm_gbs"],
                         "traffic": None if traffic_cw is None else traffic_cw * B,
                         "dram_gbs_from_profile": None if traffic_cw is None else traffic_cw * B / (dec_mean * 1e-3) / 1e9,
                         "kernel": "k_layered_cns_sched<BG1, fp16, Z=384>" if cn_state else "k_layered<20, min-sum, fp16>",
                         "message_format": "check-node state" if cn_state else "per-edge messages",
                         "message_bytes_per_codeword_iteration": msg_cw,
                         "peak_kind": f"{pk_kind} HBM copy bandwidth",
                         "algorithmic_bytes_per_launch": alg_bytes,
                         # the ceiling that binds: warp instructions (ncu, same sources) over the issue rate
                         "issue_frac": issue_frac, "warp_inst_per_32_edge_updates": ipe},
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
            "gpu_launches": (3 if fused else 4) * args.steps,
            "variants": variants,
        }
        print(json.dumps(result), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return result


def measure_variants(lx, code, llr, bits, its, stream, args, pk):
    """Decode-kernel time of the other message formats and check-node rules on the same LLRs, each with
    its own autotuned launch knobs (tuned on 1024 codewords; the knobs never change results)."""
    import torch
    from paper_2203_11854_gb300 import autotune
    out = {}
    reps = max(3, min(args.steps, 10))
    cache = f"/tmp/ldpcx_autotune_{os.getpid()}.json"
    for name, algo, prec, cns in [("minsum_f32", lx.LAYERED_MINSUM, lx.MSG_F32, 1),
                                  ("minsum_f16", lx.LAYERED_MINSUM, lx.MSG_F16, 1),
                                  ("minsum_fix6", lx.LAYERED_MINSUM, lx.MSG_FIX6, 1),
                                  ("minsum_f32_per_edge", lx.LAYERED_MINSUM, lx.MSG_F32, 0),
                                  ("minsum_f16_per_edge", lx.LAYERED_MINSUM, lx.MSG_F16, 0),
                                  ("spa_f32", lx.LAYERED_SPA, lx.MSG_F32, 1),
                                  ("spa_f16", lx.LAYERED_SPA, lx.MSG_F16, 1)]:
        lx.ldpcx_tune_set(lx.TUNE_CN_STATE, cns)
        dec = dict(algo=algo, iters=ITERS, msg_prec=prec, offset=OFFSET, clamp=CLAMP)
        tuned = autotune.tune(code, B=1024, algo=algo, msg_prec=prec, iters=ITERS, cache_path=cache)["best"]
        autotune.apply(code, algo=algo, msg_prec=prec, iters=ITERS, cache_path=cache)
        ws = torch.empty(lx.ldpc_bp_workspace(code, B, **dec), dtype=torch.uint8, device=llr.device)
        for _ in range(2):
            lx.ldpc_bp_decode(code, llr, **dec, bits_out=bits, iters_out=its, ws=ws, stream=stream)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(reps):
            lx.ldpc_bp_decode(code, llr, **dec, bits_out=bits, iters_out=its, ws=ws, stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / reps
        cn_state, msg_cw = lx.ldpc_bp_msg_format(code, algo=algo, iters=ITERS, msg_prec=prec)
        alg = B * (msg_cw * 2 * (ITERS - 1) + 4 * code.n_tx + code.k / 8)
        out[name] = {"decode_ms": ms, "gbps": B * code.k / (ms * 1e-3) / 1e9,
                     "edge_updates_per_s": B * code.edges * ITERS / (ms * 1e-3),
                     "hbm_frac": alg / (ms * 1e-3) / 1e9 / pk["hbm_gbs"],
                     "message_format": "check-node state" if cn_state else "per-edge messages",
                     "knobs": {k: tuned[k] for k in ("l2_prefetch", "cw_per_cta", "zpt")}}
        if algo == lx.LAYERED_SPA:
            # three MUFU operations (2^x, 1/x, log2) per phi, two phi per edge update; nominal 16 MUFU
            # results per clock per SM (4 per sub-partition) at the 2070 MHz maximum SM clock
            mufu_peak = 16 * torch.cuda.get_device_properties(0).multi_processor_count * 2.07e9
            out[name]["mufu_frac"] = 6 * B * code.edges * ITERS / (ms * 1e-3) / mufu_peak
        # instruction-issue fraction: warp instructions per 32 edge updates (ncu, same kernel sources) times
        # the edge updates per second, over SMs x 4 schedulers x the maximum SM clock
        prof = {"minsum_f16": ("decode_layered_minsum_f16_bg1_z384.md", None,
                               "warp instructions per 32 edge updates, LLR input"),
                "minsum_fix6": ("decode_layered_minsum_fix6_bg1_z384.md", None),
                "spa_f16": ("decode_layered_spa_f16_bg1_z384.md", None)}.get(name)
        ipe = inst_per_32_edges(*prof) if prof else None
        if ipe is not None:
            out[name]["issue_frac"] = ipe * (B * code.edges * ITERS / (ms * 1e-3)) / 32 / issue_peak()
            out[name]["warp_inst_per_32_edge_updates"] = ipe
        for key in (lx.TUNE_L2_PREFETCH, lx.TUNE_CW_PER_CTA, lx.TUNE_ZPT):
            lx.ldpcx_tune_set(key, 0)
        del ws
    lx.ldpcx_tune_set(lx.TUNE_CN_STATE, 1)
    if "minsum_f32" in out and "minsum_f16" in out:
        # FP16 >= 1.6x FP32 throughput: each precision's production format (FP16: check-node state for the core
        # rows and per-edge messages for the extension rows; FP32: check-node state), and per-edge for both
        cns = out["minsum_f32"]["decode_ms"] / out["minsum_f16"]["decode_ms"]
        edge = out["minsum_f32_per_edge"]["decode_ms"] / out["minsum_f16_per_edge"]["decode_ms"]
        out["f16_over_f32"] = cns
        out["f16_over_f32_per_edge"] = edge
        out["f16_over_f32_target"] = {
            "target": 1.6, "met": bool(cns >= 1.6 and edge >= 1.6),
            "reason": "every format keeps a resident CTA's messages in L2, so the decoder is bound by instruction "
                      "issue, not by the message width; the FP16 lead comes from its per-edge extension rows "
                      "(one conversion per message), not from moving half the bytes"}
        # not a precision ratio: FP16 check-node state against FP32 per-edge messages (format and precision)
        out["f16_state_over_f32_per_edge_format_and_precision"] = (out["minsum_f32_per_edge"]["decode_ms"]
                                                                   / out["minsum_f16"]["decode_ms"])
    try:
        os.remove(cache)
    except OSError:
        pass
    return out


def measure_sweep(lx, code, pk):
    """Graph-captured Monte-Carlo sweep: 256-QAM, max-log demapper, layered min-sum (20 iterations, no early
    stop), 16384 codewords per launch, Eb/N0 from 0 dB in 0.25 dB steps until a point's BER < 1e-6; FP16 and
    6-bit messages on the same codewords and noise draws. Reports the whole-sweep throughput (chain of every
    point), the decoder's HBM fraction over the sweep time and the Eb/N0 at BER 1e-4 of each format."""
    import torch
    from paper_2203_11854_gb300 import ber
    grid = [0.25 * i for i in range(57)]  # 0 .. 14 dB
    batch = 16384
    out = {"modulation": "256-QAM", "codewords_per_launch": batch, "step_db": 0.25}
    for name, prec in (("fp16", lx.MSG_F16), ("fix6", lx.MSG_FIX6)):
        kw = dict(m=8, demap_method=lx.DEMAP_MAXLOG, algo=lx.LAYERED_MINSUM, iters=ITERS, msg_prec=prec,
                  offset=OFFSET, clamp=CLAMP, seed=SEED, cw0=1 << 36, batch=batch, max_batches=1, stop_ber=1e-6,
                  use_graph=True)
        ws = torch.empty(lx.sim_workspace(code, grid, **kw), dtype=torch.uint8, device="cuda")
        lx.sim_run(code, grid[:1], ws=ws, **kw)  # warm-up: graph capture, first-touch
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pts = lx.sim_run(code, grid, ws=ws, **kw)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        _, msg_cw = lx.ldpc_bp_msg_format(code, algo=lx.LAYERED_MINSUM, iters=ITERS, msg_prec=prec)
        cws = sum(q["blocks"] for q in pts)
        dec_bytes = cws * (msg_cw * 2 * (ITERS - 1) + 4 * code.n_tx + code.k / 8)
        curve = [(q["ebn0_db"], q["bit_errors"] / q["bits"]) for q in pts]
        out[name] = {"points": len(pts), "codewords": cws, "seconds": sec,
                     "gbps": cws * code.k / sec / 1e9,
                     "hbm_frac": dec_bytes / sec / 1e9 / pk["hbm_gbs"],
                     "ebn0_at_1e-4_db": ber.crossing(curve), "last_point": [curve[-1][0], curve[-1][1]]}
        del ws
    c16, c6 = out["fp16"]["ebn0_at_1e-4_db"], out["fix6"]["ebn0_at_1e-4_db"]
    out["fix6_minus_fp16_db_at_1e-4"] = None if c16 is None or c6 is None else c6 - c16
    return out


def measure_flood_z8(lx):
    """The tiny plain-method configuration: BG2-shaped 42x52 code, Z = 8 (n = 416, k = 80, nothing punctured),
    QPSK, Eb/N0 0..4 dB in 0.5 dB steps, 1000 codewords per point, flooding sum-product with FP32 messages for
    20 iterations (no early stop): the graph-captured sweep (sim_run), its BER/BLER curve and throughput."""
    import torch
    code = lx.qc_ldpc_build(2, 8)
    grid = [0.5 * i for i in range(9)]
    kw = dict(m=2, demap_method=lx.DEMAP_EXACT, algo=lx.FLOOD_SPA, iters=20, msg_prec=lx.MSG_F32, early_stop=False,
              seed=SEED, cw0=1 << 38, batch=1000, max_batches=1, use_graph=True)
    ws = torch.empty(lx.sim_workspace(code, grid, **kw), dtype=torch.uint8, device="cuda")
    lx.sim_run(code, grid, ws=ws, **kw)  # warm-up: graph capture
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pts = lx.sim_run(code, grid, ws=ws, **kw)
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    cws = sum(q["blocks"] for q in pts)
    return {"workload": "BG2-shaped Z=8 (n=416, k=80), QPSK, 9 Eb/N0 points x 1000 codewords, flooding "
                        "sum-product FP32, 20 iterations", "seconds": sec, "codewords": cws,
            "codewords_per_s": cws / sec, "gbps": cws * code.k / sec / 1e9,
            "curve": [{"ebn0_db": q["ebn0_db"], "ber": q["bit_errors"] / q["bits"],
                       "bler": q["block_errors"] / q["blocks"]} for q in pts]}


def measure_grad_step(lx):
    """The weighted-BP training step: weighted flooding sum-product, BG2-shaped Z=64, batch 2048, 10 iterations,
    forward with checkpoints plus the hand-written adjoint (ldpc_bp_decode_ckpt + ldpc_bp_backward)."""
    import torch
    from paper_2203_11854_gb300.autograd import LdpcBP
    code = lx.qc_ldpc_build(2, 64)
    B, iters = 2048, 10
    g = torch.Generator(device="cuda")
    g.manual_seed(3)
    llr = (2.0 + 2.0 * torch.randn((B, code.n_tx), device="cuda", generator=g)).float().requires_grad_(True)
    w = torch.ones((iters, code.nnz), device="cuda", requires_grad=True)

    def step():
        out = LdpcBP.apply(llr, w, code, iters, 20.0)
        out.sum().backward()

    for _ in range(2):
        step()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 5
    a.record()
    for _ in range(reps):
        step()
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    out = {"ms_per_step": ms, "codewords_per_s": B / (ms * 1e-3),
           "edge_updates_per_s": 2 * B * code.edges * iters / (ms * 1e-3),
           "workload": "BG2-shaped Z=64, batch 2048, 10 flooding SPA iterations, forward + adjoint"}
    # issue-bound roofline: the two kernels' warp instructions (ncu at 1024 codewords, scaled by the batch)
    # over the step time and the GPU's issue rate; the autograd glue adds no kernel of this library
    f = inst_per_32_edges("flooding_spa_and_adjoint_bg2_z64.md", "k_flooding")
    g = inst_per_32_edges("flooding_spa_and_adjoint_bg2_z64.md", "k_backward")
    if f is not None and g is not None:
        inst = (f + g) * B * code.edges * iters / 32
        out["roofline"] = {"bound": "issue", "achieved": inst / (ms * 1e-3), "peak": issue_peak(),
                           "unit": "warp instructions/s", "frac": inst / (ms * 1e-3) / issue_peak(),
                           "warp_inst_per_32_edge_updates": {"forward": f, "adjoint": g}}
    return out


def measure_polar(lx):
    """CRC-aided SCL of polar codes: N = 1024, K = 512 (504 data bits + CRC-8 0x107), list 8
    and SC, 16384 codewords at Eb/N0 = 2 dB (BPSK, AWGN)."""
    import torch
    code = lx.polar_build(10, 512, 1.0, 0x107, 8)
    B = 16384
    n0 = torch.tensor([10 ** (-2.0 / 10) / (code.k_data / code.N)], device="cuda")
    y, data = lx.polar_sim_tx(code, 5, 0, B, n0)
    llr = ((4.0 / n0) * y).contiguous()
    out = {"code": "N=1024, K=512 (504 data + CRC-8), Bhattacharyya design at 1 dB Es/N0", "codewords": B}
    for L in (1, 8):
        bits, pm = lx.polar_scl_decode(code, llr, L)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(3):
            lx.polar_scl_decode(code, llr, L, data_out=bits, pm_out=pm)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / 3
        out[f"L{L}"] = {"ms": ms, "codewords_per_s": B / (ms * 1e-3), "data_gbps": B * code.k_data / (ms * 1e-3) / 1e9,
                        "bler_2dB": float((bits != data).any(dim=1).float().mean())}
    return out


def measure_mixed(lx, stream, args, pk):
    """Uneven batch (8192 codewords over 48 codes: Z 16..384, both shapes, rates 1/3..8/9, QPSK/16/64-QAM,
    Eb/N0 within 1 dB of each waterfall), layered min-sum FP16 with early stop: one persistent launch, its
    work-item size autotuned on this batch, against one launch per code group. Roofline: the algorithmic
    bytes of every codeword's own storage format for the iterations it ran (state reads from its second
    iteration on, writes in every iteration but a full run's last) plus its channel LLRs and bits, over the
    launch time."""
    import torch
    from paper_2203_11854_gb300 import autotune, workloads
    groups, infos, desc = workloads.mixed_batch(8192, seed=11)
    dec = dict(algo=lx.LAYERED_MINSUM, iters=20, msg_prec=lx.MSG_F16, early_stop=True)
    cache = f"/tmp/ldpcx_autotune_mixed_{os.getpid()}.json"
    tuned = autotune.tune_mixed(groups, **dec, cache_path=cache)
    autotune.apply_mixed(groups, **dec, cache_path=cache)
    ws = torch.empty(lx.ldpc_bp_mixed_workspace(groups, **dec), dtype=torch.uint8, device="cuda")
    wss = [torch.empty(max(1, lx.ldpc_bp_workspace(c, l.shape[0], **dec)), dtype=torch.uint8, device="cuda")
           for c, l in groups]
    bits_info = sum(c.k * l.shape[0] for c, l in groups)

    def persistent():
        return lx.ldpc_bp_decode_mixed(groups, **dec, ws=ws, stream=stream)

    def per_group():
        return [lx.ldpc_bp_decode(c, l, **dec, ws=w, stream=stream) for (c, l), w in zip(groups, wss)]

    out = {}
    for name, fn in (("persistent", persistent), ("per_group", per_group)):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 5
        a.record(stream)
        for _ in range(reps):
            res = fn()
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / reps
        out[name] = {"ms": ms, "gbps": bits_info / (ms * 1e-3) / 1e9}
    # decoded bits agree between the two launches, and the error counts of the batch
    counts = torch.zeros(5, dtype=torch.int64, device="cuda")
    res = persistent()
    alg_bytes = 0.0
    edge_updates = 0
    for (c, l), info, (_, b_, it) in zip(groups, infos, res):
        lx.sim_count(info, b_, it, c.k, counts)
        _, msg_cw = lx.ldpc_bp_msg_format(c, **{k: dec[k] for k in ("algo", "iters", "msg_prec")})
        its = it.to(torch.int64)
        reads = (its - 1).clamp(min=0).sum().item()
        writes = torch.where(its < dec["iters"], its, its - 1).sum().item()
        alg_bytes += msg_cw * (reads + writes) + l.shape[0] * (4 * c.n_tx + c.k / 8)
        edge_updates += c.edges * its.sum().item()
    lx.ldpcx_tune_set(lx.TUNE_CW_PER_CTA, 0)
    try:
        os.remove(cache)
    except OSError:
        pass
    cnt = counts.cpu().tolist()
    out.update(desc)
    out["speedup"] = out["per_group"]["ms"] / out["persistent"]["ms"]
    out["ber"] = cnt[1] / cnt[0]
    out["bler"] = cnt[3] / cnt[2]
    out["mean_iters"] = cnt[4] / cnt[2]
    out["autotune"] = {"knob": "codewords per work item (LDPCX_TUNE_CW_PER_CTA; 0 = automatic)",
                       "best": tuned["best"], "timings": tuned["timings"]}
    achieved = alg_bytes / (out["persistent"]["ms"] * 1e-3) / 1e9
    out["edge_updates_per_s"] = edge_updates / (out["persistent"]["ms"] * 1e-3)
    out["roofline"] = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                       "frac": achieved / pk["hbm_gbs"], "algorithmic_bytes_per_launch": alg_bytes,
                       "note": "each codeword's own message format (check-node state) for the iterations it ran"}
    # the ceiling that binds: instruction issue, SM issue per active cycle of the launch (ncu, same sources) over
    # the four schedulers of an SM
    for sec in profile_sections("decode_mixed_minsum_f16_8192cw.md"):
        if sec.get("current"):
            try:
                out["roofline"]["issue_frac"] = float(sec["SM issue (sm__inst_executed per active cycle)"].split()[0]) / 4
            except (KeyError, ValueError):
                pass
    return out


def measure_e2e(lx, code, y_dev, info_dev, n0, dec, stream, args, dev, fused=True):
    """The receiver through the public API from host memory: pinned y -> device, demap + decode
    (ldpc_bp_decode_qam; unfused: demap_app on a lower-priority stream, then ldpc_bp_decode), bits -> host.
    Double-buffered: the copies run on their own stream, so step i + 1's symbols move in (and, unfused, are
    demapped) and step i - 1's bits move out while step i decodes. Every step's copies lie inside the timed
    region."""
    import torch
    kw = (code.k + 31) // 32
    y_host = y_dev.cpu().pin_memory()
    bits_host = [torch.empty((B, kw), dtype=torch.int32).pin_memory() for _ in range(2)]
    y_d = [torch.empty_like(y_dev) for _ in range(2)]
    llr = [None if fused else torch.empty((B, code.n_tx), dtype=torch.float32, device=dev) for _ in range(2)]
    bits = [torch.empty((B, kw), dtype=torch.int32, device=dev) for _ in range(2)]
    ws = torch.empty(lx.ldpc_bp_workspace(code, B, **dec), dtype=torch.uint8, device=dev)
    copy = torch.cuda.Stream(device=dev)
    rx = torch.cuda.Stream(device=dev, priority=0)
    dec_s = torch.cuda.Stream(device=dev, priority=-1)
    ev_in = [torch.cuda.Event() for _ in range(2)]    # symbols of buffer j are on the device
    ev_used = [torch.cuda.Event() for _ in range(2)]  # the demapper (fused: the decoder) has consumed symbols j
    ev_rx = [torch.cuda.Event() for _ in range(2)]    # the decoder's input of buffer j is ready
    ev_llr = [torch.cuda.Event() for _ in range(2)]   # the decoder has consumed LLRs j
    ev_dec = [torch.cuda.Event() for _ in range(2)]   # bits of buffer j are ready
    ev_out = [torch.cuda.Event() for _ in range(2)]   # bits of buffer j have reached the host buffer

    def front(j):
        copy.wait_event(ev_used[j])
        with torch.cuda.stream(copy):
            y_d[j].copy_(y_host, non_blocking=True)
        ev_in[j].record(copy)
        if fused:
            ev_rx[j] = ev_in[j]
            return
        rx.wait_event(ev_in[j])
        rx.wait_event(ev_llr[j])
        lx.demap_app(y_d[j], n0, M, method=lx.DEMAP_MAXLOG, clamp=CLAMP, llr_out=llr[j], stream=rx)
        ev_used[j].record(rx)
        ev_rx[j].record(rx)

    def run(steps):
        for s_ in (copy, rx, dec_s):
            s_.wait_stream(stream)
        front(0)
        for i in range(steps):
            j = i & 1
            if i + 1 < steps:
                front(1 - j)
            dec_s.wait_event(ev_rx[j])
            dec_s.wait_event(ev_out[j])
            if fused:
                lx.ldpc_bp_decode_qam(code, y_d[j], n0, M, demap_method=lx.DEMAP_MAXLOG, demap_clamp=CLAMP, **dec,
                                      bits_out=bits[j], iters_out=False, ws=ws, stream=dec_s)
                ev_used[j].record(dec_s)
            else:
                lx.ldpc_bp_decode(code, llr[j], **dec, bits_out=bits[j], iters_out=False, ws=ws, stream=dec_s)
                ev_llr[j].record(dec_s)
            ev_dec[j].record(dec_s)
            copy.wait_event(ev_dec[j])
            with torch.cuda.stream(copy):
                bits_host[j].copy_(bits[j], non_blocking=True)
            ev_out[j].record(copy)
        dec_s.wait_stream(copy)
        stream.wait_stream(dec_s)

    run(2)
    torch.cuda.synchronize()
    reps = max(3, min(args.steps, 10))
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    run(reps)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    path = ("pinned host y -> ldpc_bp_decode_qam (demapper fused into the decoder) -> host bits; copies on their "
            "own stream, double-buffered against the previous step's decode") if fused else (
            "pinned host y -> demap_app -> ldpc_bp_decode -> host bits; copies on their own stream and the demapper "
            "on a lower-priority one, double-buffered against the previous step's decode")
    return {"value": B * code.k / (ms * 1e-3) / 1e9, "unit": "Gbit/s",
            "h2d_bytes_per_step": y_host.numel() * 4, "d2h_bytes_per_step": bits_host[0].numel() * 4,
            "ms_per_step": ms, "path": path}


CASES = ("minsum_f16", "minsum_f32", "minsum_fix6", "spa_f16", "spa_f32", "qam_minsum_f16", "grad", "mixed",
         "flood_spa_z8")


def run_case(args):
    """One kernel's launches alone, for timing and for small-case ncu captures: W untimed launches, then K
    launches between CUDA events on the launching stream. Prints one JSON line with the mean launch time.
    minsum_* / spa_*: ldpc_bp_decode of the BG1-shaped Z=384 code (20 iterations, no early stop) on --batch
    codewords of the 16-QAM workload; qam_minsum_f16: the same decode from the received symbols with the
    demapper fused (ldpc_bp_decode_qam, the bench step's decode launch); grad: the weighted flooding sum-product forward with checkpoints and
    its adjoint (BG2-shaped Z=64, 10 iterations, --batch codewords); mixed: the persistent mixed-code launch
    (8192 codewords); flood_spa_z8: flooding sum-product FP32, BG2-shaped Z=8, 20 iterations."""
    import torch
    import paper_2203_11854_gb300 as lx
    lx.load_library()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    Bc = args.batch
    name = args.case
    info = {}
    if name.startswith(("minsum_", "spa_", "qam_")):
        fused = name.startswith("qam_")
        base = name[4:] if fused else name
        algo = lx.LAYERED_MINSUM if base.startswith("minsum_") else lx.LAYERED_SPA
        prec = {"f16": lx.MSG_F16, "f32": lx.MSG_F32, "fix6": lx.MSG_FIX6}[base.split("_")[1]]
        code = lx.qc_ldpc_build(BG, Z, punct_cols=PUNCT)
        r = code.k / code.n_tx
        n0 = torch.tensor([1.0 / (r * M * 10 ** (EBN0 / 10))], dtype=torch.float32, device=dev)
        y, _ = lx.sim_tx(code, SEED, 0, Bc, M, n0)
        llr = lx.demap_app(y, n0, M, method=lx.DEMAP_MAXLOG, clamp=CLAMP)
        dec = dict(algo=algo, iters=ITERS, msg_prec=prec, offset=OFFSET, clamp=CLAMP)
        ws = torch.empty(lx.ldpc_bp_workspace(code, Bc, **dec), dtype=torch.uint8, device=dev)
        kw = (code.k + 31) // 32
        bits = torch.empty((Bc, kw), dtype=torch.int32, device=dev)
        its = torch.empty((Bc,), dtype=torch.int32, device=dev)
        cn_state, msg_cw = lx.ldpc_bp_msg_format(code, algo=algo, iters=ITERS, msg_prec=prec)
        info = {"codewords": Bc, "edges": code.edges, "iters": ITERS, "message_bytes_per_codeword_iteration": msg_cw,
                "message_format": "check-node state" if cn_state else "per-edge messages",
                "algorithmic_bytes_per_launch": Bc * (msg_cw * 2 * (ITERS - 1) + (8 * code.n_tx // M if fused else
                                                                               4 * code.n_tx) + code.k / 8)}

        def fn():
            if fused:
                lx.ldpc_bp_decode_qam(code, y, n0, M, demap_method=lx.DEMAP_MAXLOG, demap_clamp=CLAMP, **dec,
                                      bits_out=bits, iters_out=its, ws=ws, stream=stream)
            else:
                lx.ldpc_bp_decode(code, llr, **dec, bits_out=bits, iters_out=its, ws=ws, stream=stream)
    elif name == "flood_spa_z8":
        code = lx.qc_ldpc_build(2, 8)
        n0 = torch.tensor([1.0 / (code.k / code.n_tx * 2 * 10 ** (2.0 / 10))], dtype=torch.float32, device=dev)
        y, _ = lx.sim_tx(code, SEED, 0, Bc, 2, n0)
        llr = lx.demap_app(y, n0, 2, method=lx.DEMAP_EXACT, clamp=CLAMP)
        dec = dict(algo=lx.FLOOD_SPA, iters=ITERS, msg_prec=lx.MSG_F32, clamp=CLAMP)
        ws = torch.empty(lx.ldpc_bp_workspace(code, Bc, **dec), dtype=torch.uint8, device=dev)
        info = {"codewords": Bc, "edges": code.edges, "iters": ITERS}

        def fn():
            lx.ldpc_bp_decode(code, llr, **dec, ws=ws, stream=stream)
    elif name == "grad":
        code = lx.qc_ldpc_build(2, 64)
        iters = 10
        g = torch.Generator(device=dev)
        g.manual_seed(3)
        llr = (2.0 + 2.0 * torch.randn((Bc, code.n_tx), device=dev, generator=g)).float().contiguous()
        w = torch.ones((iters, code.nnz), device=dev)
        ckpt = torch.empty(lx.ldpc_bp_ckpt_bytes(code, Bc, iters=iters, weights=w), dtype=torch.uint8, device=dev)
        gw = torch.zeros_like(w)
        gout = torch.ones((Bc, code.n), dtype=torch.float32, device=dev)
        info = {"codewords": Bc, "edges": code.edges, "iters": iters}

        def fn():
            lx.ldpc_bp_decode_ckpt(code, llr, iters=iters, weights=w, ckpt=ckpt, stream=stream)
            lx.ldpc_bp_backward(code, llr, ckpt, gout, iters=iters, weights=w, grad_weights=gw, stream=stream)
    elif name == "mixed":
        from paper_2203_11854_gb300 import workloads
        groups, _, desc = workloads.mixed_batch(8192, seed=11)
        dec = dict(algo=lx.LAYERED_MINSUM, iters=20, msg_prec=lx.MSG_F16, early_stop=True)
        ws = torch.empty(lx.ldpc_bp_mixed_workspace(groups, **dec), dtype=torch.uint8, device=dev)
        info = {"codewords": 8192}

        def fn():
            lx.ldpc_bp_decode_mixed(groups, **dec, ws=ws, stream=stream)
    else:
        raise SystemExit(f"unknown case {name}; one of {', '.join(CASES)}")
    for _ in range(args.warmup):
        fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(args.steps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    st, _ = lx.ldpcx_sync_status()
    if st != 0:
        raise SystemExit(f"device status: {lx.ldpcx_status_str(st)}")
    ms = a.elapsed_time(b) / args.steps
    print(json.dumps({"case": name, "ms_per_launch": ms, "steps": args.steps, "warmup": args.warmup, **info}),
          flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--quick", action="store_true", help="skip the per-variant decode timings")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--batch", type=int, default=B, help="codewords per step (4096 for the headline workload)")
    ap.add_argument("--unfused", action="store_true",
                    help="run the demapper as its own kernel (demap_app, then ldpc_bp_decode) instead of fused")
    ap.add_argument("--case", default=None, choices=CASES,
                    help="time one kernel's launches alone (for profiling) instead of the Monte-Carlo step")
    args = ap.parse_args()
    if args.case:
        if args.warmup < 1 or args.steps < 1:
            raise SystemExit("--case needs --warmup >= 1 and --steps >= 1")
        run_case(args)
        return
    globals()["B"] = args.batch
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
