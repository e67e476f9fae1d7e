#!/usr/bin/env python3
"""Benchmark of the LSB embed/extract hot path on one 8192x8192x3 uint8
cover (201,326,592 bytes) carrying a message at full one-bit capacity
(25,165,820 bytes behind the 32-bit header).

One step = one embed (with the fused changed-byte/SSE count) and one
extract of that cover, inputs resident in HBM.  The L2 (129 MB) is flushed
before each timed call (a 256 MiB write, then a 512 MiB read so no dirty
line is left); the flushes sit outside the timed intervals, which CUDA
events on the launching stream measure.
value = cover bytes processed (2 per step: the embed and the extract each
traverse the cover once) / device time, summed over ranks for N > 1 (each
rank runs its own replica; no data-path collective).

Prints one JSON line.  `--impl reference` times the CPU oracle instead (on
the host cores, rank 0 only) on the same workload, cut to a prefix only if
the whole cover would not fit the time budget.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cover GB/s embed/extract vs HBM peak; batched vs per-image launch; p99 latency"
UNIT = "cover GB/s"
L2_FLUSH_BYTES = 256 << 20
FALLBACK_HBM_GBS = 6800.0

# DRAM traffic per launch of the embed kernels (dram__bytes_read.sum +
# dram__bytes_write.sum) from one ncu capture on this exact workload, per
# kernel family, valid only while the kernel sources hash to `src_sha`.
# Writes still dirty in the L2 when the kernel exits are not in the count.
NCU_TRAFFIC = {"embed_vec": {"src_sha": "95a135be69318ee7", "bytes": 226519296 + 144900096},
               "embed_bulk": {"src_sha": "c5b02751867fd4e8", "bytes": 226599680 + 142849024}}
# The same counters for one launch in the middle of the steady-state
# sequence (back-to-back launches over distinct buffers, no flush; ncu with
# --cache-control none): the previous launches' deferred write-backs land in
# it as its own do in the next ones, so it counts one launch's full traffic.
NCU_TRAFFIC_STEADY = {"embed_vec": {"src_sha": "95a135be69318ee7",
                                    "bytes": 226511360 + 200450048}}
KERNEL_SOURCES = ("s1_device.cuh", "stream1.cu", "bulk.cu", "internal.cuh")
MAX_RING = 192 * 1024


def staged_stages(t) -> int:
    """Stages of the shared-memory staged kernels for a single-cover shape
    (0: the register kernels run), as the library derives them."""
    if not t.tile_bytes:
        return 0
    tile = t.threads * 16 * t.vec_per_thread
    st = min(8, t.tile_bytes // tile)
    while st >= 2 and st * tile > MAX_RING:
        st -= 1
    return st if st >= 2 else 0


def embed_kernel_name(t) -> tuple[str, str]:
    fam = "embed_bulk" if staged_stages(t) else "embed_vec"
    return fam, "%s<%d,true>" % (fam, t.vec_per_thread)


def kernel_src_sha() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_0912_0947_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            v = float(json.load(f)["hbm_gbs"])
        return v, "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while running."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if r[4 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ----------------------------------------------------------------------------
# multi-rank aggregation (replicas: every rank runs its own cover)
# ----------------------------------------------------------------------------

def max_over_ranks(value: float, world: int, device) -> float:
    """The largest per-rank value (the slowest rank bounds the job); a
    timing reduction only, no data moves between ranks."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(bytes_per_rank: float, max_ms: float, world: int) -> float:
    """Whole-job GB/s: the bytes every rank processed over the slowest rank's
    time."""
    return world * bytes_per_rank / (max_ms / 1e3) / 1e9


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------

def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_0912_0947_gb300 as S
    from paper_0912_0947_gb300 import autotune as AT, build as B, synth

    if not os.path.exists(B.LIB):
        raise RuntimeError("libstego.so missing: run __graft_entry__.build() first")
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    w = synth.single_8192()
    C, m = w.cover_bytes, w.msg_bytes
    cover = w.cover(dev)
    msg = w.message(dev)
    stego = torch.empty_like(cover)
    out = torch.empty(m, dtype=torch.uint8, device=dev)
    res_e = S.new_result(dev)
    res_x = S.new_result(dev)
    flush = AT.Flusher(dev, L2_FLUSH_BYTES)
    fe = S.HEADER_BE32 | S.FUSE_STATS
    fx = S.HEADER_BE32
    stream = torch.cuda.current_stream(dev)

    def embed():
        S.stego_embed(cover, stego, msg, fe, res_e, stream=stream)

    def extract():
        S.stego_extract(stego, out, 0, fx, res_x, stream=stream)

    tuning = {}
    fixed = {"embed": args.shape_embed, "extract": args.shape_extract}
    embed()
    for name, op, fn in (("embed", S.OP_EMBED, embed), ("extract", S.OP_EXTRACT, extract)):
        if fixed[name]:
            S.stego_set_tune(op, tuple(int(x) for x in fixed[name].split(",")))
            tuning[name] = {"fixed": fixed[name]}
        elif not args.no_tune:
            best, us, table = AT.autotune(op, fn, C, flush=flush, use_cache=False)
            staged = [t for s_, t in table if s_[3]]
            tuning[name] = {"best": list(best), "us": round(us, 2), "candidates": len(table),
                            "worst_us": round(max(t for _, t in table), 2),
                            "best_register_us": round(min(t for s_, t in table if not s_[3]), 2),
                            "best_staged_us": round(min(staged), 2) if staged else None}

    if args.profile_case:
        return run_profile_case(S, torch, dev, synth, args.profile_case)
    if args.steady_only:
        return {"steady_only": run_steady_leg(S, torch, dev, stream, cover, msg, C, m,
                                              max(args.steady_pairs, 2)),
                "launch": {"embed": tune_dict(S.stego_get_tune(S.OP_EMBED)),
                           "extract": tune_dict(S.stego_get_tune(S.OP_EXTRACT))}}

    def step(ev=None):
        flush()
        if ev:
            ev[0].record(stream)
        embed()
        if ev:
            ev[1].record(stream)
        flush()
        if ev:
            ev[2].record(stream)
        extract()
        if ev:
            ev[3].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    # correctness of the timed configuration (the parity tests cover the rest)
    r = S.read_result(res_x)
    assert r["status"] == 0 and r["msg_bytes"] == m and torch.equal(out, msg)

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    sampler = ClockSampler(local_rank) if rank == 0 else None
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    if sampler:
        sampler.start()
        time.sleep(0.3)
    t_wall0 = time.perf_counter()
    for k in range(args.steps):
        step(evs[k])
    torch.cuda.synchronize(dev)
    t_wall = time.perf_counter() - t_wall0
    if world > 1:
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    t_emb = [evs[k][0].elapsed_time(evs[k][1]) for k in range(args.steps)]  # ms
    t_ext = [evs[k][2].elapsed_time(evs[k][3]) for k in range(args.steps)]
    dev_ms = max_over_ranks(sum(t_emb) + sum(t_ext), world, dev)
    value = job_throughput(2.0 * C * args.steps, dev_ms, world)

    stats = S.read_result(res_e)
    # ---- practical roofline: a same-size device copy, timed the same way ---
    copy = None
    if rank == 0:
        t_copy = AT.time_call(lambda: stego.copy_(cover), flush, 20, stream=stream)
        embed()  # restore the stego
        copy_gbs = 2 * C / (t_copy * 1e-6) / 1e9
        copy = {"what": "torch copy_ of the %d-byte cover into the stego buffer (2C bytes), "
                        "L2 flushed, median of 20" % C,
                "us": round(t_copy, 2), "gbs": round(copy_gbs, 1)}
    # ---- steady state: back-to-back launches over distinct buffers ----------
    steady = None
    if rank == 0 and args.steady_pairs > 0:
        steady = run_steady_leg(S, torch, dev, stream, cover, msg, C, m, args.steady_pairs)
        torch.cuda.empty_cache()
    # ---- end to end through the public API with host buffers ---------------
    e2e = None
    if (rank == 0 or world > 1) and args.e2e_steps > 0:
        e2e = run_e2e_library(args, S, torch, dev, cover, msg, C, m)
        e2e["zero_copy_host_stego"] = run_e2e_zero_copy(args, S, torch, dev, stream, cover,
                                                        msg, C, m)
        e2e["explicit_copy"] = run_e2e(args, S, torch, dev, stream, cover, msg, C, m)
    # ---- batched vs one launch per image -----------------------------------------
    legs = {}
    uneven_tune = None  # the uneven batch's tuned batched shapes, for its other legs
    if world > 1 and not args.no_batched:
        # every rank takes part: the 4096-cover batch split by byte volume
        sharded = run_sharded_leg(S, AT, torch, dev, stream, synth, rank, world,
                                  count=args.uneven_count or None)
        if sharded:
            legs["batched_uneven_sharded"] = sharded
        torch.cuda.empty_cache()
    if world > 1 or not args.legs or "split_cover" in args.legs.split(","):
        # every rank takes part: the one cover split at 16-byte offsets
        split = run_split_leg(S, AT, torch, dev, stream, rank, world, cover, stego, msg, C, m)
        if split:
            legs["split_cover"] = split
        torch.cuda.empty_cache()
    single_gpu_legs = {"batched_uneven", "batched_video", "batched_video_paper2", "paper2",
                       "streamk", "serving", "small", "extract_gather", "batched_uneven_host",
                       "batched_uneven_misaligned", "single_misaligned"}
    # with several GPUs the run is the replicated step and the two splits
    # above; the one-GPU legs are the N = 1 run's (the other GPUs would idle
    # while rank 0 repeated them)
    want = set(args.legs.split(",")) if args.legs else (single_gpu_legs if world == 1 else set())
    if args.no_batched:
        want -= {"batched_uneven", "batched_video", "batched_video_paper2", "paper2", "streamk",
                 "batched_uneven_host", "batched_uneven_misaligned"}
    if args.no_serving:
        want.discard("serving")
    del flush
    torch.cuda.empty_cache()
    for kind in ("uneven", "video", "video_paper2"):
        if rank == 0 and "batched_" + kind in want:
            legs["batched_" + kind] = run_batched_leg(
                S, AT, torch, dev, stream, synth, kind,
                count=(args.uneven_count if kind == "uneven" else args.video_frames) or None,
                tune=not args.no_tune)
            if kind == "uneven" and legs[("batched_" + kind)]["launch"]:
                sel = legs["batched_uneven"]["launch"]
                uneven_tune = (tuple(sel["embed"]), tuple(sel["extract"]))
            torch.cuda.empty_cache()
    if rank == 0 and "streamk" in want:
        legs["streamk"] = run_streamk_leg(S, AT, torch, dev, synth)
        torch.cuda.empty_cache()
    if rank == 0 and "extract_gather" in want:
        legs["extract_gather"] = run_extract_gather_leg(S, AT, torch, dev, synth)
        torch.cuda.empty_cache()
    if rank == 0 and "single_misaligned" in want:
        legs["single_misaligned"] = run_misaligned_leg(S, AT, torch, dev, synth)
        torch.cuda.empty_cache()
    if rank == 0 and "small" in want:
        legs["small_512x512x3"] = run_small_leg(S, AT, torch, dev, synth)
        torch.cuda.empty_cache()
    if rank == 0 and "paper2" in want:
        legs["paper2"] = run_paper2_leg(S, AT, torch, dev, synth)
        torch.cuda.empty_cache()
    if rank == 0 and "batched_uneven_misaligned" in want:
        legs["batched_uneven_misaligned"] = run_misaligned_batched_leg(
            S, AT, torch, dev, stream, synth, count=args.uneven_count or None, tune=uneven_tune)
        torch.cuda.empty_cache()
    if rank == 0 and "batched_uneven_host" in want:
        legs["batched_uneven_host"] = run_host_batched_leg(S, torch, dev, synth,
                                                           count=args.uneven_count or None,
                                                           tune=uneven_tune)
        torch.cuda.empty_cache()
    if rank == 0 and "serving" in want:
        legs["serving"] = run_serving_leg(S, AT, torch, dev, synth,
                                          [1000, 2000, 5000, 10000, 20000, 50000],
                                          max_requests=args.serving_max_requests,
                                          seconds=args.serving_seconds)
        torch.cuda.empty_cache()
    # ---- CPU oracle baseline ----------------------------------------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cover_h, msg_h = cover.cpu().numpy(), msg.cpu().numpy()
        embed()  # the timed configuration's outputs, compared with the oracle's
        extract()
        torch.cuda.synchronize(dev)
        cpu = run_cpu_baseline(cover_h, msg_h, budget_s=args.cpu_seconds,
                               gpu_stego=stego.cpu().numpy(), gpu_msg=out.cpu().numpy())
        cpu["all_cores"] = run_cpu_all_cores(cover_h, msg_h, budget_s=args.cpu_seconds / 2)

    if rank != 0:
        return None
    peak, peak_kind = hbm_peak()
    T = 8 * (m + 4)
    emb_bytes = 2 * C + T // 8
    ext_bytes = T + T // 8
    emb_us = statistics.mean(t_emb) * 1e3
    ext_us = statistics.mean(t_ext) * 1e3
    achieved = emb_bytes / (emb_us * 1e-6) / 1e9
    sha = kernel_src_sha()
    t_emb_shape = S.stego_get_tune(S.OP_EMBED)
    fam, kname = embed_kernel_name(t_emb_shape)
    rec = NCU_TRAFFIC.get(fam)
    traffic = rec["bytes"] if rec and rec["src_sha"] == sha else None
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dev_ms / args.steps, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u8", "data": "synthetic",
        "config": {
            "workload": "single 8192x8192x3 uint8 cover, full 1-bit capacity "
                        "(25165820 B message + 32-bit header); embed (fused stats) + extract",
            "cover_bytes": C, "msg_bytes": m, "carrying_bytes": T,
            "l2": "flushed before each timed call, outside the timed interval: write 256 MiB, "
                  "then read 512 MiB so no dirty line is left for the timed call, then a "
                  "100k-cycle GPU spin so the call is queued before its start event runs",
            "parallelism": "replicas" if world > 1 else "single GPU",
            "launch": {"embed": tune_dict(S.stego_get_tune(S.OP_EMBED)),
                       "extract": tune_dict(S.stego_get_tune(S.OP_EXTRACT))},
            "autotune": tuning,
        },
        "embed": {"us": round(emb_us, 2), "cover_gbs": round(C / (emb_us * 1e-6) / 1e9, 1),
                  "algorithmic_bytes": emb_bytes,
                  "hbm_frac": round(achieved / peak, 4)},
        "extract": {"us": round(ext_us, 2), "cover_gbs": round(C / (ext_us * 1e-6) / 1e9, 1),
                    "algorithmic_bytes": ext_bytes,
                    "hbm_frac": round(ext_bytes / (ext_us * 1e-6) / 1e9 / peak, 4)},
        "roofline": {"bound": "hbm", "kernel": kname + " (stego_embed, fused stats)",
                     "stages": staged_stages(t_emb_shape),
                     "achieved": round(achieved, 1), "peak": peak, "peak_kind": peak_kind,
                     "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "traffic": traffic,
                     "regime": "L2 flushed before the launch, write-back deferred: stego "
                               "lines still dirty in the L2 when the kernel ends reach DRAM "
                               "after the timed interval (the ncu traffic counts only what "
                               "was written back during the launch)",
                     "note": "achieved = (2C + T/8) bytes / mean event time of the stego_embed "
                             "call (one kernel launch: the statistics go through the "
                             "stream's accumulator slot, no zeroing copy)"},
        "copy_roofline": dict(copy, embed_frac_of_copy=round(achieved / copy["gbs"], 4),
                              extract_frac_of_copy=round(
                                  ext_bytes / (ext_us * 1e-6) / 1e9 / copy["gbs"], 4))
        if copy else None,
        "psnr_db": round(10.0 * __import__("math").log10(255.0 ** 2 * C / stats["sse"]), 4)
        if stats["sse"] else None,
        "gpu_launches": 2 * args.steps,
        "wall_ms_per_step_incl_flush": round(t_wall * 1e3 / args.steps, 4),
        "clocks": clocks,
    }
    if steady:
        st_emb = emb_bytes / (steady["embed_us"] * 1e-6) / 1e9
        st_ext = ext_bytes / (steady["extract_us"] * 1e-6) / 1e9
        rec_s = NCU_TRAFFIC_STEADY.get(fam)
        line["roofline"].update({
            "achieved_steady": round(st_emb, 1), "frac_steady": round(st_emb / peak, 4),
            "traffic_steady": rec_s["bytes"] if rec_s and rec_s["src_sha"] == sha else None,
            "steady": dict(steady, embed_frac=round(st_emb / peak, 4),
                           extract_frac=round(st_ext / peak, 4),
                           embed_frac_of_copy=round(st_emb / steady["copy_gbs"], 4),
                           regime="steady state: back-to-back launches, every write-back "
                                  "inside the timed interval")})
    if e2e:
        line["e2e"] = e2e
    line.update(legs)
    if cpu:
        line["cpu_baseline"] = cpu
    return line


def run_batched_leg(S, AT, torch, dev, stream, synth, kind, count=None, tune=True):
    """Many covers in one batched launch (and its CUDA-graph replay) against
    one stego_embed / stego_extract launch per cover, same bytes, same GPU.

    uneven: 4096 covers, sides log-uniform in [64, 4096], 1 or 3 channels,
            messages filling 5..100 % of capacity;
    video:  600 frames of 1920x1080x3, gradient plus noise, one message
            stream split across frames at half capacity, header per frame."""
    paper = kind == "video_paper2"
    if kind == "uneven":
        items = synth.uneven_batch(count or 4096)
        sizes = [it.cover_bytes for it in items]
        mlens = [it.msg_bytes for it in items]
    else:
        v = synth.Video(frames=count or 600)
        sizes = [v.frame_bytes] * v.frames
        mlens = [v.per_frame_msg] * v.frames
    n = len(sizes)
    off, moff, p, q = [], [], 0, 0
    for c, m in zip(sizes, mlens):
        off.append(p)
        moff.append(q)
        p += (c + 255) // 256 * 256
        q += (m + 255) // 256 * 256
    if kind == "uneven":
        covers = synth.uniform_bytes(p, synth.substream(synth.SEED_BASE + 4, 1), dev)
        msgs = synth.uniform_bytes(q, synth.substream(synth.SEED_BASE + 4, 2), dev)
    else:
        covers = torch.empty(p, dtype=torch.uint8, device=dev)
        for f0 in range(0, n, 50):
            fr = v.frame_range(f0, min(n, f0 + 50), dev).view(-1, v.frame_bytes)
            for i in range(fr.shape[0]):
                covers[off[f0 + i]: off[f0 + i] + v.frame_bytes] = fr[i]
            del fr
        stream_msg = v.message(dev)
        msgs = torch.zeros(q, dtype=torch.uint8, device=dev)
        P = v.per_frame_msg
        for f in range(n):
            msgs[moff[f]: moff[f] + P] = stream_msg[f * P:(f + 1) * P]
        del stream_msg
    stego_b = torch.empty_like(covers)
    stego_1 = torch.empty_like(covers)
    out_b = torch.empty_like(msgs)
    out_1 = torch.empty_like(msgs)
    cv = [covers[o:o + c] for o, c in zip(off, sizes)]
    sb = [stego_b[o:o + c] for o, c in zip(off, sizes)]
    s1 = [stego_1[o:o + c] for o, c in zip(off, sizes)]
    mv = [msgs[o:o + m] for o, m in zip(moff, mlens)]
    ob = [out_b[o:o + m] for o, m in zip(moff, mlens)]
    o1 = [out_1[o:o + m] for o, m in zip(moff, mlens)]
    hdr = S.LAYOUT_PAPER2 if paper else S.HEADER_BE32
    geo = dict(width=v.width, height=v.height, channels=3, plane=0) if paper else {}
    geom = (v.width, v.height, 3, 0) if paper else None
    d_emb = S.descs_to_device(S.pack_descs(
        [dict(cover=cv[i], stego=sb[i], msg=mv[i], cover_bytes=sizes[i], msg_bytes=mlens[i],
              flags=hdr, **geo) for i in range(n)]), dev)
    d_ext = S.descs_to_device(S.pack_descs(
        [dict(cover=sb[i], msg=ob[i], cover_bytes=sizes[i], msg_bytes=mlens[i],
              msg_len=mlens[i], flags=hdr, **geo) for i in range(n)]), dev)
    res_b = S.new_result(dev, n=n)
    res_1 = S.new_result(dev, n=n)
    res_x1 = S.new_result(dev, n=n)
    ws = torch.empty(S.stego_batched_workspace_bytes(n), dtype=torch.uint8, device=dev)
    flush = AT.Flusher(dev)

    def b_embed():
        S.stego_embed_batched(d_emb, n, res_b, S.FUSE_STATS, ws, stream=stream)

    def b_extract():
        S.stego_extract_batched(d_ext, n, res_b, 0, ws, stream=stream)

    def one_embed():
        for i in range(n):
            S.stego_embed(cv[i], s1[i], mv[i], hdr | S.FUSE_STATS, res_1[i], geom=geom,
                          stream=stream)

    def one_extract():
        for i in range(n):
            S.stego_extract(s1[i], o1[i], mlens[i], hdr, res_x1[i], geom=geom, stream=stream)

    tune_sel = {}
    for name, op, fn in (("embed", S.OP_EMBED_BATCHED, b_embed),
                         ("extract", S.OP_EXTRACT_BATCHED, b_extract)):
        if tune:
            best, us, table = AT.autotune(op, fn, p, flush=flush, reps=5, use_cache=False)
            tune_sel[name] = list(best)
    t_be = AT.time_call(b_embed, flush, 7)
    t_bx = AT.time_call(b_extract, flush, 7)
    t_1e = AT.time_call(one_embed, flush, 3)
    t_1x = AT.time_call(one_extract, flush, 3)
    # graph replay of the batched embed (same descriptors, results, workspace)
    g = S.BatchedGraph(S.OP_EMBED_BATCHED, d_emb, n, res_b, S.FUSE_STATS, ws)
    t_ge = AT.time_call(lambda: g.launch(stream), flush, 7)
    g.close()
    b_extract()
    torch.cuda.synchronize()
    # compare cover by cover (the 256-byte padding between slots is never written)
    same = all(torch.equal(sb[i], s1[i]) and torch.equal(ob[i], o1[i]) for i in range(n))
    assert same, "batched and per-image outputs differ"
    assert all(torch.equal(ob[i], mv[i]) for i in range(n)), "batched round trip differs"
    extra = {}
    if kind != "uneven":
        # in place (stego == cover): re-embedding the same message is idempotent
        inpl = covers.clone()
        iv = [inpl[o:o + c] for o, c in zip(off, sizes)]
        d_inp = S.descs_to_device(S.pack_descs(
            [dict(cover=iv[i], stego=iv[i], msg=mv[i], cover_bytes=sizes[i],
                  msg_bytes=mlens[i], flags=hdr, **geo) for i in range(n)]), dev)
        t_bi = AT.time_call(lambda: S.stego_embed_batched(d_inp, n, res_b, S.FUSE_STATS, ws,
                                                          stream=stream), flush, 7)
        torch.cuda.synchronize()
        assert all(torch.equal(iv[i], sb[i]) for i in range(n)), "in-place batched differs"
        extra["embed_in_place_batched_us"] = round(t_bi, 1)
        del inpl, iv, d_inp
    else:
        # the same covers as separate allocations (one tensor per cover,
        # message and output) instead of slots of one arena
        sc = [x.clone() for x in cv]
        ss = [torch.empty_like(x) for x in sc]
        sm = [x.clone() for x in mv]
        so = [torch.empty_like(x) for x in sm]
        d_se = S.descs_to_device(S.pack_descs(
            [dict(cover=sc[i], stego=ss[i], msg=sm[i], cover_bytes=sizes[i],
                  msg_bytes=mlens[i], flags=hdr) for i in range(n)]), dev)
        d_sx = S.descs_to_device(S.pack_descs(
            [dict(cover=ss[i], msg=so[i], cover_bytes=sizes[i], msg_bytes=mlens[i],
                  flags=hdr) for i in range(n)]), dev)
        t_se = AT.time_call(lambda: S.stego_embed_batched(d_se, n, res_b, S.FUSE_STATS, ws,
                                                          stream=stream), flush, 7)
        t_sx = AT.time_call(lambda: S.stego_extract_batched(d_sx, n, res_b, 0, ws,
                                                            stream=stream), flush, 7)
        torch.cuda.synchronize()
        assert all(torch.equal(ss[i], sb[i]) and torch.equal(so[i], mv[i]) for i in range(n)), \
            "separate-tensor batched differs"
        extra["separate_tensors"] = {"embed_batched_us": round(t_se, 1),
                                     "extract_batched_us": round(t_sx, 1)}
        del sc, ss, sm, so
    total = sum(sizes)
    if paper:  # out of place 2C + N; extraction touches every sector of its rows
        emb_bytes = sum(2 * c + m for c, m in zip(sizes, mlens))
        rows = [-(-m // (v.width // 4)) for m in mlens]
        ext_bytes = sum(r * v.width * 3 + m for r, m in zip(rows, mlens))
        # in place: the carrying plane bytes' sectors of the carrying rows
        inp_bytes = sum(2 * r * v.width * 3 + m for r, m in zip(rows, mlens))
    else:
        T = [8 * (m + 4) for m in mlens]
        emb_bytes = sum(2 * c + t // 8 for c, t in zip(sizes, T))
        ext_bytes = sum(t + t // 8 for t in T)
        inp_bytes = sum(2 * t + t // 8 for t in T)
    peak, _ = hbm_peak()
    gbs = lambda b, us: round(b / (us * 1e-6) / 1e9, 1)
    if "embed_in_place_batched_us" in extra:
        t_bi = extra["embed_in_place_batched_us"]
        extra["embed_in_place"] = {"algorithmic_bytes": inp_bytes,
                                   "cover_gbs": gbs(total, t_bi),
                                   "hbm_frac": round(inp_bytes / (t_bi * 1e-6) / 1e9 / peak, 4)}
    if "separate_tensors" in extra:
        st_ = extra["separate_tensors"]
        st_["embed_cover_gbs"] = gbs(total, st_["embed_batched_us"])
        st_["extract_cover_gbs"] = gbs(total, st_["extract_batched_us"])
    return {
        "workload": ("4096 uneven covers (log-uniform sides 64..4096, 1 or 3 channels, "
                     "5-100% fill)" if kind == "uneven" else
                     ("%d frames 1920x1080x3, gradient+noise, paper layout (plane 0, 2 bits/byte), "
                      "388796 message bytes per frame" % n) if paper else
                     "%d frames 1920x1080x3, gradient+noise, half capacity per frame" % n),
        "covers": n, "cover_bytes": total,
        "embed_batched_us": round(t_be, 1), "embed_graph_us": round(t_ge, 1),
        "embed_per_image_us": round(t_1e, 1),
        "extract_batched_us": round(t_bx, 1), "extract_per_image_us": round(t_1x, 1),
        "embed_cover_gbs": {"batched": gbs(total, t_be), "graph": gbs(total, t_ge),
                            "per_image": gbs(total, t_1e)},
        "extract_cover_gbs": {"batched": gbs(total, t_bx), "per_image": gbs(total, t_1x)},
        "speedup_batched_vs_per_image": {"embed": round(t_1e / t_be, 2),
                                         "extract": round(t_1x / t_bx, 2)},
        "hbm_frac_batched": {"embed": round(emb_bytes / (t_be * 1e-6) / 1e9 / peak, 4),
                             "extract": round(ext_bytes / (t_bx * 1e-6) / 1e9 / peak, 4)},
        "launch": tune_sel,
        "outputs_identical": same,
        **extra,
    }


def run_misaligned_batched_leg(S, AT, torch, dev, stream, synth, count=None, tune=None):
    """The 4096-cover uneven batch with every cover 1..15 bytes past a
    16-byte boundary and every stego at its own random offset (the funnel
    routine: stego vectors joined from cover vector pairs; same offsets take
    the shift routine), messages at random parity, against the same batch in
    256-byte aligned slots; outputs compared with the aligned batch's."""
    items = synth.uneven_batch(count or 4096)
    sizes = [it.cover_bytes for it in items]
    mlens = [it.msg_bytes for it in items]
    n = len(sizes)
    import numpy as np
    rng = np.random.default_rng(7)
    coff = [int(x) for x in rng.integers(1, 16, n)]
    soff = [int(x) for x in rng.integers(1, 16, n)]
    moff = [int(x) for x in rng.integers(0, 2, n)]

    def layout(offs, lens, pad):
        pos, p = [], 0
        for o, c in zip(offs, lens):
            pos.append(p + o)
            p += (c + pad + 255) // 256 * 256
        return pos, p

    cpos, pc = layout(coff, sizes, 16)
    spos, ps = layout(soff, sizes, 16)
    mpos, pm = layout(moff, mlens, 2)
    apos, pa = layout([0] * n, sizes, 0)
    bpos, pb = layout([0] * n, mlens, 0)
    covers = torch.empty(pc, dtype=torch.uint8, device=dev)
    msgs = torch.empty(pm, dtype=torch.uint8, device=dev)
    acov = synth.uniform_bytes(pa, synth.substream(synth.SEED_BASE + 4, 1), dev)
    amsg = synth.uniform_bytes(pb, synth.substream(synth.SEED_BASE + 4, 2), dev)
    for i in range(n):
        covers[cpos[i]:cpos[i] + sizes[i]] = acov[apos[i]:apos[i] + sizes[i]]
        msgs[mpos[i]:mpos[i] + mlens[i]] = amsg[bpos[i]:bpos[i] + mlens[i]]
    stego = torch.empty(ps, dtype=torch.uint8, device=dev)
    astego = torch.empty_like(acov)
    out = torch.empty(pm, dtype=torch.uint8, device=dev)
    aout = torch.empty_like(amsg)
    cv = [covers[cpos[i]:cpos[i] + sizes[i]] for i in range(n)]
    sv = [stego[spos[i]:spos[i] + sizes[i]] for i in range(n)]
    mv = [msgs[mpos[i]:mpos[i] + mlens[i]] for i in range(n)]
    ov = [out[mpos[i]:mpos[i] + mlens[i]] for i in range(n)]
    acv = [acov[apos[i]:apos[i] + sizes[i]] for i in range(n)]
    asv = [astego[apos[i]:apos[i] + sizes[i]] for i in range(n)]
    amv = [amsg[bpos[i]:bpos[i] + mlens[i]] for i in range(n)]
    aov = [aout[bpos[i]:bpos[i] + mlens[i]] for i in range(n)]
    pk = lambda c, s_, m_: S.descs_to_device(S.pack_descs(
        [dict(cover=c[i], stego=s_[i], msg=m_[i], cover_bytes=sizes[i], msg_bytes=mlens[i],
              flags=S.HEADER_BE32) for i in range(n)]), dev)
    px = lambda st_, o_: S.descs_to_device(S.pack_descs(
        [dict(cover=st_[i], msg=o_[i], cover_bytes=sizes[i], msg_bytes=mlens[i],
              flags=S.HEADER_BE32) for i in range(n)]), dev)
    d_me, d_mx = pk(cv, sv, mv), px(sv, ov)
    d_ae, d_ax = pk(acv, asv, amv), px(asv, aov)
    res = S.new_result(dev, n=n)
    ws = torch.empty(S.stego_batched_workspace_bytes(n), dtype=torch.uint8, device=dev)
    flush = AT.Flusher(dev)
    te_, tx_ = tune if tune else (None, None)
    emb = lambda d: S.stego_embed_batched(d, n, res, S.FUSE_STATS, ws, tune=te_, stream=stream)
    ext = lambda d: S.stego_extract_batched(d, n, res, 0, ws, tune=tx_, stream=stream)
    t = {"misaligned_embed_us": AT.time_call(lambda: emb(d_me), flush, 7),
         "aligned_embed_us": AT.time_call(lambda: emb(d_ae), flush, 7),
         "misaligned_extract_us": AT.time_call(lambda: ext(d_mx), flush, 7),
         "aligned_extract_us": AT.time_call(lambda: ext(d_ax), flush, 7)}
    torch.cuda.synchronize(dev)
    same = all(torch.equal(sv[i], asv[i]) and torch.equal(ov[i], mv[i]) for i in range(n))
    assert same, "misaligned batched outputs differ from the aligned batch's"
    total = sum(sizes)
    T = [8 * (m + 4) for m in mlens]
    emb_bytes = sum(2 * c + t_ // 8 for c, t_ in zip(sizes, T))
    ext_bytes = sum(t_ + t_ // 8 for t_ in T)
    peak, _ = hbm_peak()
    frac = lambda b, us: round(b / (us * 1e-6) / 1e9 / peak, 4)
    return {"workload": "4096 uneven covers as in batched_uneven, each cover 1..15 bytes past "
                        "a 16-byte boundary, each stego at its own random offset 1..15, "
                        "messages at random parity",
            "covers": n, "cover_bytes": total,
            "launch": {"embed": te_, "extract": tx_},
            **{k: round(v, 1) for k, v in t.items()},
            "hbm_frac": {"misaligned_embed": frac(emb_bytes, t["misaligned_embed_us"]),
                         "aligned_embed": frac(emb_bytes, t["aligned_embed_us"]),
                         "misaligned_extract": frac(ext_bytes, t["misaligned_extract_us"]),
                         "aligned_extract": frac(ext_bytes, t["aligned_extract_us"])},
            "misaligned_over_aligned": {
                "embed": round(t["misaligned_embed_us"] / t["aligned_embed_us"], 3),
                "extract": round(t["misaligned_extract_us"] / t["aligned_extract_us"], 3)},
            "outputs_identical_to_aligned": same}


def run_sharded_leg(S, AT, torch, dev, stream, synth, rank, world, count=None):
    """The 4096-cover uneven batch split among the ranks by byte volume
    (stego_partition): every rank embeds (fused statistics) and extracts its
    own covers in one batched launch each; no data crosses between GPUs and
    only the per-cover results are gathered on the host afterwards.  Each
    timed call starts after a barrier; the time is the slowest rank's."""
    import torch.distributed as dist

    from paper_0912_0947_gb300 import shard
    items = synth.uneven_batch(count or 4096)
    sizes = [it.cover_bytes for it in items]
    mlens = [it.msg_bytes for it in items]
    n = len(sizes)
    off, moff, p, q = [], [], 0, 0
    for c, m in zip(sizes, mlens):
        off.append(p)
        moff.append(q)
        p += (c + 255) // 256 * 256
        q += (m + 255) // 256 * 256
    # every rank generates the same arena and works on its own covers
    covers = synth.uniform_bytes(p, synth.substream(synth.SEED_BASE + 4, 1), dev)
    msgs = synth.uniform_bytes(q, synth.substream(synth.SEED_BASE + 4, 2), dev)
    stego = torch.empty_like(covers)
    out = torch.zeros_like(msgs)
    mine = shard.my_covers(sizes, rank, world)
    k = len(mine)
    d_e = S.descs_to_device(S.pack_descs(
        [dict(cover=covers[off[i]:off[i] + sizes[i]], stego=stego[off[i]:off[i] + sizes[i]],
              msg=msgs[moff[i]:moff[i] + mlens[i]], cover_bytes=sizes[i], msg_bytes=mlens[i],
              flags=S.HEADER_BE32) for i in mine]), dev)
    d_x = S.descs_to_device(S.pack_descs(
        [dict(cover=stego[off[i]:off[i] + sizes[i]], msg=out[moff[i]:moff[i] + mlens[i]],
              cover_bytes=sizes[i], msg_bytes=mlens[i], flags=S.HEADER_BE32) for i in mine]), dev)
    res_e = S.new_result(dev, n=max(k, 1))
    res_x = S.new_result(dev, n=max(k, 1))
    ws = torch.empty(S.stego_batched_workspace_bytes(max(k, 1)), dtype=torch.uint8, device=dev)
    flush = AT.Flusher(dev)

    def timed(fn, reps=5):
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize(dev)
            dist.barrier()
            flush()  # ends in a short GPU spin: the call is queued before e0 runs
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ts.append(max_over_ranks(e0.elapsed_time(e1), world, dev))
        return sorted(ts)[len(ts) // 2]

    emb = lambda: S.stego_embed_batched(d_e, k, res_e, S.FUSE_STATS, ws, stream=stream) if k else None
    ext = lambda: S.stego_extract_batched(d_x, k, res_x, 0, ws, stream=stream) if k else None
    emb()
    ext()
    t_e = timed(emb)
    t_x = timed(ext)
    re = S.read_result(res_e)[:k] if k else []
    rx = S.read_result(res_x)[:k] if k else []
    ok_local = all(r["status"] == 0 for r in re + rx) and all(
        torch.equal(out[moff[i]:moff[i] + mlens[i]], msgs[moff[i]:moff[i] + mlens[i]])
        for i in mine)
    gathered = shard.gather_results(mine, [(r["status"], r["changed"], r["sse"]) for r in re], n)
    oks = [None] * world
    dist.all_gather_object(oks, ok_local)
    _, rank_bytes = S.stego_partition(sizes, world)
    total = sum(sizes)
    if rank != 0:
        return None
    assert all(oks) and all(g is not None and g[0] == 0 for g in gathered),         "sharded batch failed"
    return {"workload": "4096 uneven covers as in batched_uneven, split among %d GPUs by byte "
                        "volume (stego_partition), one batched launch per GPU" % world,
            "ranks": world, "cover_bytes": total,
            "rank_cover_bytes": [int(b) for b in rank_bytes],
            "imbalance_bytes": int(rank_bytes.max() - rank_bytes.min()),
            "largest_cover_bytes": max(sizes),
            "embed_ms_slowest_rank": round(t_e, 3), "extract_ms_slowest_rank": round(t_x, 3),
            "embed_cover_gbs": round(total / (t_e * 1e-3) / 1e9, 1),
            "extract_cover_gbs": round(total / (t_x * 1e-3) / 1e9, 1),
            "scaling": "strong (the same 4096 covers split among the GPUs)",
            "gathered_changed": int(sum(g[1] for g in gathered))}


def run_split_leg(S, AT, torch, dev, stream, rank, world, cover, stego, msg, C, m):
    """The 8192x8192x3 cover at full capacity split among the ranks at
    16-byte cover offsets (shard.cover_slices): every rank embeds (fused
    statistics) and extracts only its own slice, reading the header from
    the first 32 stego bytes like a rank without the message length would.
    With one process the slice is the whole cover (the split's own cost:
    the header's four bytes go through a call of their own).  Each timed
    call starts after a barrier; the time is the slowest rank's."""
    from paper_0912_0947_gb300 import shard
    c0, c1 = shard.cover_slices(C, world)[rank]
    lo, hi = shard.slice_message_range(c0, c1, m)
    cs, part = cover[c0:c1], msg[lo:hi]
    st = torch.empty(c1 - c0, dtype=torch.uint8, device=dev)
    out = torch.empty(max(hi - lo, 1), dtype=torch.uint8, device=dev)
    head = stego[:32]  # rank 0's first stego bytes, written by the single-cover embed
    flush = AT.Flusher(dev)

    mm = shard.read_header(head, C, stream=stream)
    emb_sl = shard.CoverSlice(c0, c1, C, m, device=dev)
    ext_sl = shard.CoverSlice(c0, c1, C, mm, device=dev)

    def emb():
        emb_sl.embed(cs, st, part, stream=stream)

    def ext():
        ext_sl.extract(st, out, stream=stream)

    def timed(fn, reps=9):
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize(dev)
            if world > 1:
                import torch.distributed as dist
                dist.barrier()
            flush()  # ends in a short GPU spin: the calls are queued before e0 runs
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ts.append(max_over_ranks(e0.elapsed_time(e1), world, dev))
        return sorted(ts)[len(ts) // 2]

    emb()
    ext()
    torch.cuda.synchronize(dev)
    ok = (mm == m and torch.equal(st, stego[c0:c1]) and torch.equal(out[: hi - lo], part))
    ch, ss = emb_sl.stats(stream)
    t_e = timed(emb)
    t_x = timed(ext)
    oks = [ok]
    if world > 1:
        import torch.distributed as dist
        oks = [None] * world
        dist.all_gather_object(oks, (ok, ch))
        oks = [o[0] for o in oks]
    if rank != 0:
        return None
    assert all(oks), "split cover differs from the single-cover embed"
    return {"workload": "8192x8192x3 cover (201,326,592 B) at full one-bit capacity split among "
                        "%d GPUs at 16-byte cover offsets, one slice per GPU" % world,
            "ranks": world, "slice_bytes": [b - a for a, b in shard.cover_slices(C, world)],
            "embed_ms_slowest_rank": round(t_e, 4), "extract_ms_slowest_rank": round(t_x, 4),
            "embed_cover_gbs": round(C / (t_e * 1e-3) / 1e9, 1),
            "extract_cover_gbs": round(C / (t_x * 1e-3) / 1e9, 1),
            "header_read": "once per cover before the timed extractions: the header's 4 "
                           "bytes extracted from the first 32 stego bytes and read back",
            "scaling": "strong (one cover split among the GPUs)"}


# launch shape of the server's batched calls: the library's built-in
# batched default (threads, vectors per thread, CTAs per SM, tile bytes)
SERVING_TUNE = (256, 4, 0, 65536)


def run_serving_leg(S, AT, torch, dev, synth, rates, max_requests=1000000, seconds=20.0,
                    saturation_rates=(100000, 200000, 500000, 1000000, 2000000, 3000000,
                                      5000000)):
    """Open-loop Poisson request stream against the continuous-batching
    server: 70% embed / 30% extract over a resident pool of 4096 uneven covers
    (sizes as in the batched leg) and their pre-embedded stegos, messages and
    outputs resident on the device, 40 GB in-flight budget.  Each offered
    rate runs `seconds` of arrivals (at most max_requests); after the listed
    rates the offered rate keeps rising until the server no longer keeps up
    (throughput under 90% of the offered rate): the knee."""
    import numpy as np
    items = synth.uneven_batch(4096)
    sizes = [it.cover_bytes for it in items]
    mlens = [it.msg_bytes for it in items]
    n = len(sizes)
    off, moff, p, q = [], [], 0, 0
    for c, m in zip(sizes, mlens):
        off.append(p)
        moff.append(q)
        p += (c + 255) // 256 * 256
        q += (m + 255) // 256 * 256
    covers = synth.uniform_bytes(p, synth.substream(synth.SEED_BASE + 5, 1), dev)
    msgs = synth.uniform_bytes(q, synth.substream(synth.SEED_BASE + 5, 2), dev)
    stegos = torch.empty_like(covers)
    out_st = torch.empty_like(covers)
    out_msg = torch.empty_like(msgs)
    ws = torch.empty(S.stego_batched_workspace_bytes(n), dtype=torch.uint8, device=dev)
    d = S.descs_to_device(S.pack_descs(
        [dict(cover=covers[off[i]:off[i] + sizes[i]], stego=stegos[off[i]:off[i] + sizes[i]],
              msg=msgs[moff[i]:moff[i] + mlens[i]], cover_bytes=sizes[i], msg_bytes=mlens[i],
              flags=S.HEADER_BE32) for i in range(n)]), dev)
    S.stego_embed_batched(d, n, S.new_result(dev, n=n), 0, ws)  # the resident stegos
    torch.cuda.synchronize()
    base = {"cover": covers.data_ptr(), "stego": stegos.data_ptr(), "out_st": out_st.data_ptr(),
            "msg": msgs.data_ptr(), "out_msg": out_msg.data_ptr()}
    off_a = np.array(off, dtype=np.uint64)
    moff_a = np.array(moff, dtype=np.uint64)
    size_a = np.array(sizes, dtype=np.uint64)
    mlen_a = np.array(mlens, dtype=np.uint64)
    results = []
    embedded, extracted = set(), set()
    total_batches = 0

    def one_rate(ri, rate):
        cnt = int(min(max_requests, max(500, rate * seconds)))
        u = synth.uniform_floats_np(2 * cnt, synth.substream(synth.SEED_BASE + 5, 100 + ri))
        ids = np.minimum((u[:cnt] * n).astype(np.int64), n - 1)
        is_ext = u[cnt:] < 0.3
        reqs = np.zeros(cnt, dtype=S.REQUEST_DTYPE)
        o, mo, cb, mb = off_a[ids], moff_a[ids], size_a[ids], mlen_a[ids]
        reqs["op"] = np.where(is_ext, S.OP_EXTRACT, S.OP_EMBED)
        reqs["flags"] = S.HEADER_BE32
        reqs["cover"] = np.where(is_ext, base["stego"] + o, base["cover"] + o)
        reqs["stego"] = np.where(is_ext, 0, base["out_st"] + o)
        reqs["msg"] = np.where(is_ext, base["out_msg"] + mo, base["msg"] + mo)
        reqs["cover_bytes"] = cb
        reqs["msg_bytes"] = mb
        arr = synth.poisson_arrivals(float(rate), cnt,
                                     synth.substream(synth.SEED_BASE + 5, 200 + ri))
        # the library's default batched shapes, whatever earlier legs installed
        srv = S.Server(slots=8, max_batch=512, budget_bytes=40 << 30, device=dev,
                       tune_embed=SERVING_TUNE, tune_extract=SERVING_TUNE)
        comps = srv.run_open_loop(reqs, arr, timeout_s=600)
        stats = srv.stats()
        srv.close()
        embedded.update(int(i) for i in ids[~is_ext][:64])
        extracted.update(int(i) for i in ids[is_ext][:64])
        assert np.all(comps["status"] == 0), "serving requests failed"
        lat = (comps["t_done"] - comps["t_submit"]) * 1e3
        span = float(comps["t_done"].max() - comps["t_submit"].min())
        return {
            "offered_req_per_s": rate, "requests": cnt,
            "arrival_span_s": round(float(arr[-1]), 3),
            "throughput_req_per_s": round(cnt / span, 1),
            "cover_gbs": round(float(cb.sum()) / span / 1e9, 2),
            "p50_ms": round(float(np.percentile(lat, 50)), 4),
            "p99_ms": round(float(np.percentile(lat, 99)), 4),
            "max_ms": round(float(lat.max()), 4),
            "mean_batch": round(float(comps["batch_size"].mean()), 2),
            "batches": stats["batches"],
            "peak_in_flight_bytes": stats["peak_in_flight_bytes"],
        }

    for ri, rate in enumerate(rates):
        results.append(one_rate(ri, rate))
    knee = None
    for k, rate in enumerate(saturation_rates):
        r = one_rate(len(rates) + k, rate)
        results.append(r)
        if r["throughput_req_per_s"] < 0.9 * rate:
            knee = r
            break
    # served outputs equal single calls (a sample of the covers embedded)
    for i in sorted(embedded)[:64]:
        ref = torch.empty(sizes[i], dtype=torch.uint8, device=dev)
        S.stego_embed(covers[off[i]:off[i] + sizes[i]], ref, msgs[moff[i]:moff[i] + mlens[i]],
                      S.HEADER_BE32)
        assert torch.equal(ref, out_st[off[i]:off[i] + sizes[i]])
    for i in sorted(extracted)[:64]:
        assert torch.equal(out_msg[moff[i]:moff[i] + mlens[i]], msgs[moff[i]:moff[i] + mlens[i]])
    kept = [r for r in results if r["throughput_req_per_s"] >= 0.9 * r["offered_req_per_s"]]
    return {"workload": "Poisson open loop, 70% embed / 30% extract, 4096 resident uneven "
                        "covers and stegos, 40 GB in-flight budget, 8 slots, batches <= 512",
            "launch": {"embed": SERVING_TUNE, "extract": SERVING_TUNE},
            "per_rate": "max(500, min(%d, rate x %g s)) requests, a new server per rate" % (
                max_requests, seconds),
            "rates": results,
            "max_sustained": kept[-1] if kept else None,
            "knee": knee if knee else {"note": "no saturation up to %d req/s" % saturation_rates[-1]}}


def run_paper2_leg(S, AT, torch, dev, synth):
    """The paper's own layout (Sections VI/VII) on the 8192x8192x3 cover:
    plane 0, two bits per byte, floor(W/4)*H = 16,777,216 message bytes (full
    capacity).  Algorithmic bytes: out of place 2C + N; in place 2*4N + N
    (carrying plane bytes); extract 4N + N.  The plane bytes are every third
    byte, so DRAM moves whole 32-byte sectors: in place and extract touch
    every sector of the cover (about 2C + N and C + N)."""
    W = H = 8192
    C, N = W * H * 3, (W // 4) * H
    cover = synth.uniform_bytes(C, synth.substream(synth.SEED_BASE + 6, 1), dev)
    msg = synth.uniform_bytes(N, synth.substream(synth.SEED_BASE + 6, 2), dev)
    stego = torch.empty_like(cover)
    buf = torch.empty_like(cover)
    out = torch.empty(N, dtype=torch.uint8, device=dev)
    res = S.new_result(dev)
    geom = (W, H, 3, 0)
    flush = AT.Flusher(dev)
    fl = S.LAYOUT_PAPER2 | S.FUSE_STATS

    def oop():
        S.stego_embed(cover, stego, msg, fl, res, geom=geom)

    def inplace():
        S.stego_embed(buf, buf, msg, fl, res, geom=geom)

    def ext():
        S.stego_extract(stego, out, N, S.LAYOUT_PAPER2, res, geom=geom)

    t_o = AT.time_call(oop, flush, 15)
    buf.copy_(cover)
    t_i = AT.time_call(inplace, flush, 15)
    t_x = AT.time_call(ext, flush, 15)
    torch.cuda.synchronize()
    assert torch.equal(out, msg) and torch.equal(buf, stego)
    peak, _ = hbm_peak()
    g = lambda b, us: round(b / (us * 1e-6) / 1e9, 1)
    return {
        "workload": "8192x8192x3 cover, plane 0, 2 bits/byte, 16777216-byte message (full capacity)",
        "embed_out_of_place_us": round(t_o, 2), "embed_in_place_us": round(t_i, 2),
        "extract_us": round(t_x, 2),
        "cover_gbs": {"embed_out_of_place": g(C, t_o), "embed_in_place": g(C, t_i),
                      "extract": g(C, t_x)},
        "hbm_frac": {"embed_out_of_place": round(g(2 * C + N, t_o) / peak, 4),
                     "embed_in_place_sectors": round(g(2 * C + N, t_i) / peak, 4),
                     "extract_sectors": round(g(C + N, t_x) / peak, 4)},
        "algorithmic_bytes": {"embed_out_of_place": 2 * C + N, "embed_in_place": 9 * N,
                              "extract": 5 * N},
    }


def run_streamk_leg(S, AT, torch, dev, synth):
    """The stream layout with k bits per carrying byte on the 8192x8192x3
    cover at full capacity: k = 2, 3 and 4 over all bytes (algorithmic bytes
    2C + 8|S|/8 embed, C + |S| extract) and k = 2 on plane 0 (carrying bytes
    every third byte: sectors of the whole cover move)."""
    C = 8192 * 8192 * 3
    cover = synth.uniform_bytes(C, synth.substream(synth.SEED_BASE + 7, 1), dev)
    stego = torch.empty_like(cover)
    res = S.new_result(dev)
    flush = AT.Flusher(dev)
    peak, _ = hbm_peak()
    out = {}
    for name, k, geom in (("k2_all", 2, None), ("k3_all", 3, None), ("k4_all", 4, None),
                          ("k2_plane0", 2, (8192, 8192, 3, 0))):
        flags = S.BITS(k) | S.HEADER_BE32 | (S.PLANE_ONLY if geom else 0)
        m = S.stego_capacity(C, flags, geom=geom)
        msg = synth.uniform_bytes(m, synth.substream(synth.SEED_BASE + 7, 10 + k), dev)
        got = torch.empty(m, dtype=torch.uint8, device=dev)

        def emb():
            S.stego_embed(cover, stego, msg, flags | S.FUSE_STATS, res, geom=geom)

        def ext():
            S.stego_extract(stego, got, 0, flags, res, geom=geom)

        te = AT.time_call(emb, flush, 15)
        tx = AT.time_call(ext, flush, 15)
        torch.cuda.synchronize()
        assert torch.equal(got, msg)
        s_bytes = m + 4
        carry = -(-8 * s_bytes // k) * (3 if geom else 1)  # cover bytes spanned by the carriers
        eb = 2 * C + s_bytes
        xb = min(carry, C) + s_bytes
        out[name] = {"msg_bytes": m, "embed_us": round(te, 2), "extract_us": round(tx, 2),
                     "embed_cover_gbs": round(C / (te * 1e-6) / 1e9, 1),
                     "extract_cover_gbs": round(C / (tx * 1e-6) / 1e9, 1),
                     "embed_hbm_frac": round(eb / (te * 1e-6) / 1e9 / peak, 4),
                     "extract_hbm_frac": round(xb / (tx * 1e-6) / 1e9 / peak, 4)}
        del msg, got
    return out


def run_extract_gather_leg(S, AT, torch, dev, synth,
                           shapes=((128, 4, 0, 0), (256, 4, 0, 0), (512, 4, 0, 0),
                                   (128, 4, 8, 0), (256, 2, 4, 0), (512, 8, 2, 0))):
    """The full-capacity 8192x8192x3 extraction by the vector kernel
    (stego_extract: 16 stego bytes per lane, one multiply per four bytes)
    and by the ballot kernel (stego_extract_ballot: one stego byte per lane,
    one ballot per message word), same launch shapes, L2 flushed."""
    w = synth.single_8192()
    cover, msg = w.cover(dev), w.message(dev)
    stego = torch.empty_like(cover)
    S.stego_embed(cover, stego, msg, S.HEADER_BE32)
    out = torch.empty(w.msg_bytes, dtype=torch.uint8, device=dev)
    res = S.new_result(dev)
    flush = AT.Flusher(dev)
    old = S.stego_get_tune(S.OP_EXTRACT)
    table = []
    try:
        for sh in shapes:
            S.stego_set_tune(S.OP_EXTRACT, sh)
            tv = AT.time_call(lambda: S.stego_extract(stego, out, 0, S.HEADER_BE32, res), flush, 15)
            tb = AT.time_call(lambda: S.stego_extract_ballot(stego, out, 0, S.HEADER_BE32, res),
                              flush, 15)
            table.append((list(sh[:3]), round(tv, 2), round(tb, 2)))
        torch.cuda.synchronize()
        assert torch.equal(out, msg)
    finally:
        S.stego_set_tune(S.OP_EXTRACT, old)
    T = 8 * (w.msg_bytes + 4)
    peak, _ = hbm_peak()
    bv, bb = min(t[1] for t in table), min(t[2] for t in table)
    frac = lambda us: round((T + T // 8) / (us * 1e-6) / 1e9 / peak, 4)
    return {"workload": "8192x8192x3 cover, full one-bit capacity, header extraction",
            "vector_best_us": bv, "ballot_best_us": bb,
            "hbm_frac": {"vector": frac(bv), "ballot": frac(bb)},
            "shapes_vector_ballot_us": table}


def run_small_leg(S, AT, torch, dev, synth, reps=25, burst=1000):
    """The 512x512x3 cover (786,432 bytes) with a 32,768-byte message behind
    the header: the whole working set fits the L2, so the time is launch and
    latency bound.  Cold = L2 flushed before each call, warm = after an
    untimed run of the same call (both with the call queued before its start
    event); back to back = `burst` calls between two events (device time per
    call, launch gaps included); enqueue = host time per API call;
    graph = one embed + one extract captured in a CUDA graph, replayed back
    to back (device time per pair)."""
    w = synth.single_512()
    C, m = w.cover_bytes, w.msg_bytes
    cover, msg = w.cover(dev), w.message(dev)
    stego = torch.empty_like(cover)
    out = torch.empty(m, dtype=torch.uint8, device=dev)
    res_e, res_x = S.new_result(dev), S.new_result(dev)
    stream = torch.cuda.current_stream(dev)
    flush = AT.Flusher(dev)

    def emb():
        S.stego_embed(cover, stego, msg, S.HEADER_BE32 | S.FUSE_STATS, res_e, stream=stream)

    def ext():
        S.stego_extract(stego, out, 0, S.HEADER_BE32, res_x, stream=stream)

    r = {"workload": "512x512x3 uint8 cover, 32768-byte message + 32-bit header "
                     "(T = 262176 carrying bytes)"}
    for name, fn in (("embed", emb), ("extract", ext)):
        fn()
        cold = AT.time_call(fn, flush, reps, stream=stream)

        def warm_up(fn=fn):  # the same call untimed (its data now in L2), then a spin
            fn()
            torch.cuda._sleep(AT.SPIN_CYCLES)

        warm = AT.time_call(fn, warm_up, reps, stream=stream)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(stream)
        for _ in range(burst):
            fn()
        e1.record(stream)
        t_host = time.perf_counter() - t0
        torch.cuda.synchronize(dev)
        b2b = e0.elapsed_time(e1) * 1e3 / burst
        r[name] = {"cold_us": round(cold, 2), "warm_us": round(warm, 2),
                   "back_to_back_us": round(b2b, 2),
                   "enqueue_us": round(t_host * 1e6 / burst, 2),
                   "cover_gbs_cold": round(C / (cold * 1e-6) / 1e9, 1),
                   "cover_gbs_back_to_back": round(C / (b2b * 1e-6) / 1e9, 1)}
    assert torch.equal(out, msg)
    # one embed + one extract captured into a CUDA graph, replayed back to back
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream(dev)
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        emb_s = lambda: S.stego_embed(cover, stego, msg, S.HEADER_BE32 | S.FUSE_STATS, res_e,
                                      stream=side)
        ext_s = lambda: S.stego_extract(stego, out, 0, S.HEADER_BE32, res_x, stream=side)
        emb_s()
        ext_s()
    torch.cuda.synchronize(dev)
    with torch.cuda.graph(g, stream=side):
        emb_s()
        ext_s()
    out.zero_()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(burst):
        g.replay()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    assert torch.equal(out, msg)
    r["graph_embed_extract_us"] = round(e0.elapsed_time(e1) * 1e3 / burst, 2)
    return r


def run_steady_leg(S, torch, dev, stream, cover, msg, C, m, pairs, rounds=5):
    """The timed embed and extract launched back to back, with no flush in
    between, over `pairs` distinct cover/stego/message sets (pairs x 427 MB,
    far more than the 129 MB L2): each launch's stego writes that are still
    dirty in the L2 when it ends are written back while the next launches
    run, inside the timed interval, so the mean launch time is the steady
    state.  One event interval around all pairs x rounds launches."""
    covers = [cover.clone() for _ in range(pairs)]
    msgs = [msg.clone() for _ in range(pairs)]
    stegos = [torch.empty_like(cover) for _ in range(pairs)]
    outs = [torch.empty_like(msg) for _ in range(pairs)]
    res = S.new_result(dev, n=pairs)
    fe, fx = S.HEADER_BE32 | S.FUSE_STATS, S.HEADER_BE32

    def emb(k):
        S.stego_embed(covers[k], stegos[k], msgs[k], fe, res[k], stream=stream)

    def ext(k):
        S.stego_extract(stegos[k], outs[k], 0, fx, res[k], stream=stream)

    out = {}
    for name, fn in (("embed", emb), ("extract", ext)):
        for k in range(pairs):  # warm-up, and the stegos for the extract
            fn(k)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(rounds):
            for k in range(pairs):
                fn(k)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        out[name + "_us"] = round(e0.elapsed_time(e1) * 1e3 / (rounds * pairs), 2)
    # the same back-to-back sequence as a plain device copy of each cover
    # into its stego (torch copy_, 2C bytes per launch): the practical
    # ceiling of a read + write stream in this regime
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for k in range(pairs):
        stegos[k].copy_(covers[k])
    e0.record(stream)
    for _ in range(rounds):
        for k in range(pairs):
            stegos[k].copy_(covers[k])
    e1.record(stream)
    torch.cuda.synchronize(dev)
    out["copy_us"] = round(e0.elapsed_time(e1) * 1e3 / (rounds * pairs), 2)
    out["copy_gbs"] = round(2 * C / (out["copy_us"] * 1e-6) / 1e9, 1)
    for k in range(pairs):  # the stegos again, for the round-trip check
        emb(k)
        ext(k)
    torch.cuda.synchronize(dev)
    rr = S.read_result(res)
    assert all(r["status"] == 0 and r["msg_bytes"] == m for r in rr)
    assert all(torch.equal(o, msg) for o in outs), "steady-state round trip differs"
    out.update({"pairs": pairs, "launches": rounds * pairs,
                "what": "back-to-back launches over %d distinct 8192x8192x3 cover/stego/message "
                        "sets (%.1f GB), no flush between them; one event interval" % (
                            pairs, pairs * (2 * C + m) / 1e9)})
    return out


MISALIGNED_CASES = ((0, 0, 0), (3, 3, 0), (5, 5, 1), (3, 7, 0), (0, 8, 0), (12, 4, 1))


def misaligned_views(S, torch, dev, w, co, so, mo):
    """The 8192x8192x3 cover (less 16 bytes) and its message placed co, so
    and mo bytes past 256-byte aligned allocations: cover, stego and
    message at those misalignments, the message at full capacity."""
    C, m = w.cover_bytes, w.msg_bytes
    Cm = C - 16
    mm = Cm // 8 - 4
    bufs = [torch.empty(C + 64, dtype=torch.uint8, device=dev) for _ in range(2)] + \
        [torch.empty(m + 64, dtype=torch.uint8, device=dev) for _ in range(2)]
    cv, sv = bufs[0][co:co + Cm], bufs[1][so:so + Cm]
    mv, ov = bufs[2][mo:mo + mm], bufs[3][mo:mo + mm]
    cv.copy_(w.cover(dev)[:Cm])
    mv.copy_(w.message(dev)[:mm])
    return bufs, cv, sv, mv, ov, Cm, mm


def run_misaligned_leg(S, AT, torch, dev, synth):
    """Single-cover embed (fused statistics) and extract of the 201 MB cover
    with the cover, stego and message at several misalignments (cover
    offset, stego offset, message offset from a 16-byte boundary): same
    offset (vectors after a scalar head), different offsets (stego vectors
    joined from cover vector pairs), and the extract of a misaligned stego;
    each against the aligned case, outputs compared with it."""
    w = synth.single_8192()
    flush = AT.Flusher(dev)
    peak, _ = hbm_peak()
    res = S.new_result(dev)
    ref = None
    out = {}
    for co, so, mo in MISALIGNED_CASES:
        bufs, cv, sv, mv, ov, Cm, mm = misaligned_views(S, torch, dev, w, co, so, mo)
        fe = lambda: S.stego_embed(cv, sv, mv, S.HEADER_BE32 | S.FUSE_STATS, res)
        fx = lambda: S.stego_extract(sv, ov, 0, S.HEADER_BE32, res)
        te = AT.time_call(fe, flush, 15)
        tx = AT.time_call(fx, flush, 15)
        torch.cuda.synchronize(dev)
        if ref is None:
            ref = sv.clone()
        assert torch.equal(sv, ref) and torch.equal(ov, mv), "misaligned outputs differ"
        T = 8 * (mm + 4)
        out["c%d_s%d_m%d" % (co, so, mo)] = {
            "embed_us": round(te, 2), "embed_frac": round((2 * Cm + T // 8) / (te * 1e-6) / 1e9
                                                          / peak, 4),
            "extract_us": round(tx, 2), "extract_frac": round((T + T // 8) / (tx * 1e-6) / 1e9
                                                              / peak, 4)}
        del bufs
    return {"workload": "8192x8192x3 cover less 16 bytes at full capacity; key c<cover>_s<stego>"
                        "_m<message> = byte offsets from a 16-byte boundary", "cases": out}


def run_profile_case(S, torch, dev, synth, spec):
    """--profile-case co,so,mo: one warm-up and one more embed + extract of
    the misaligned case; --profile-case kK: the same with k bits over every
    byte of the aligned cover at full capacity (for a profiler)."""
    if spec.startswith("k"):
        k = int(spec[1:])
        w = synth.single_8192()
        cover = w.cover(dev)
        flags = S.BITS(k) | S.HEADER_BE32
        m = S.stego_capacity(cover.numel(), flags)
        msg = synth.uniform_bytes(m, synth.substream(synth.SEED_BASE + 7, 10 + k), dev)
        stego, got = torch.empty_like(cover), torch.empty_like(msg)
        res = S.new_result(dev)
        for _ in range(2):
            S.stego_embed(cover, stego, msg, flags | S.FUSE_STATS, res)
            S.stego_extract(stego, got, 0, flags, res)
        torch.cuda.synchronize(dev)
        assert torch.equal(got, msg)
        return {"profile_case": spec, "ok": True}
    co, so, mo = (int(x) for x in spec.split(","))
    w = synth.single_8192()
    bufs, cv, sv, mv, ov, Cm, mm = misaligned_views(S, torch, dev, w, co, so, mo)
    res = S.new_result(dev)
    for _ in range(2):
        S.stego_embed(cv, sv, mv, S.HEADER_BE32 | S.FUSE_STATS, res)
        S.stego_extract(sv, ov, 0, S.HEADER_BE32, res)
    torch.cuda.synchronize(dev)
    assert torch.equal(ov, mv)
    return {"profile_case": spec, "ok": True}


def tune_dict(t):
    return {"threads": t.threads, "vec_per_thread": t.vec_per_thread,
            "ctas_per_sm": t.ctas_per_sm, "tile_bytes": t.tile_bytes}


def run_e2e_zero_copy(args, S, torch, dev, stream, cover_d, msg_d, C, m):
    """The step through the public API on host buffers: the cover, message,
    stego and extracted message live in pinned host memory and the kernels
    read and write them directly over the CPU-GPU link (no staging copy);
    each call's 32-byte result is read back to the host."""
    cover_h = cover_d.cpu().pin_memory()
    msg_h = msg_d.cpu().pin_memory()
    stego_h = torch.empty(C, dtype=torch.uint8).pin_memory()
    out_h = torch.empty(m, dtype=torch.uint8).pin_memory()
    res_h = torch.empty(4, dtype=torch.int64).pin_memory()
    res2_h = torch.empty(4, dtype=torch.int64).pin_memory()
    r_d = S.new_result(dev)
    r2_d = S.new_result(dev)

    def step():
        S.stego_embed(cover_h, stego_h, msg_h, S.HEADER_BE32 | S.FUSE_STATS, r_d, stream=stream)
        res_h.copy_(r_d, non_blocking=True)
        S.stego_extract(stego_h, out_h, 0, S.HEADER_BE32, r2_d, stream=stream)
        res2_h.copy_(r2_d, non_blocking=True)

    for _ in range(2):
        step()
    torch.cuda.synchronize(dev)
    assert torch.equal(out_h, msg_h) and int(res2_h[2]) == m
    n = args.e2e_steps
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(n):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / n
    return {"value": round(2.0 * C / (ms * 1e-3) / 1e9, 2), "unit": UNIT,
            "ms_per_step": round(ms, 4), "steps": n, "mode": "zero-copy (pinned host buffers)",
            "h2d_bytes_per_step": 2 * C + m, "d2h_bytes_per_step": C + m + 64}


def run_e2e_library(args, S, torch, dev, cover_d, msg_d, C, m, slots=3):
    """The step through the library's host pipeline (stego_pipeline_embed):
    every step is one host-resident job -- the cover and message are copied
    from pinned host memory into a device slot, embedded there (fused
    statistics), the new stego is extracted on the device (the job's
    read-back), and the stego and the extracted message are copied back to
    pinned host memory.  The pipeline runs neighbouring steps' copy-in,
    kernels and copy-out at the same time on its own three streams; the
    timed region is the whole synchronous call over all steps (host wall
    clock), so every input and output byte crosses the link inside it."""
    cover_h = cover_d.cpu().pin_memory()
    msg_h = msg_d.cpu().pin_memory()
    stego_h = torch.empty(C, dtype=torch.uint8).pin_memory()
    out_h = torch.empty(m, dtype=torch.uint8).pin_memory()
    # one job per slot: cover, message and read-back plus the placement slack
    pipe = S.Pipeline(slots=slots, max_descs=1, slot_bytes=C + m + (m + 255) // 256 * 256 + 1280)
    job = dict(cover=cover_h, stego=stego_h, msg=msg_h, readback=out_h, cover_bytes=C,
               msg_bytes=m, flags=S.HEADER_BE32)
    n = args.e2e_steps
    jobs = S.Pipeline.jobs([job] * n)
    res, rb = pipe.embed(S.Pipeline.jobs([job] * slots), S.FUSE_STATS, readback_results=True)
    assert all(r["status"] == 0 for r in res + rb)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    res, rb = pipe.embed(jobs, S.FUSE_STATS, readback_results=True)
    ms = (time.perf_counter() - t0) * 1e3 / n
    pipe.close()
    assert all(r["status"] == 0 and r["msg_bytes"] == m for r in res + rb)
    want = torch.empty_like(cover_d)
    S.stego_embed(cover_d, want, msg_d, S.HEADER_BE32)
    torch.cuda.synchronize(dev)
    assert torch.equal(stego_h, want.cpu()), "pipelined stego differs"
    assert torch.equal(out_h, msg_h), "pipelined read-back differs"
    return {"value": round(2.0 * C / (ms * 1e-3) / 1e9, 2), "unit": UNIT,
            "ms_per_step": round(ms, 4), "steps": n,
            "api": "stego_pipeline_embed (%d slots), one host job per step with a read-back "
                   "extraction; host wall clock around the call" % slots,
            "h2d_bytes_per_step": C + m + 72, "d2h_bytes_per_step": C + m + 64}


def run_host_batched_leg(S, torch, dev, synth, count=None, slots=3, slot_mb=256, tune=None):
    """The 4096 uneven covers of the batched leg held in pinned host memory
    (cover, stego and message arenas), embedded and then extracted through
    the library's host pipeline: copy-in, batched kernels and copy-out of
    neighbouring chunks overlapped.  Host wall clock around each call."""
    items = synth.uneven_batch(count or 4096)
    sizes = [it.cover_bytes for it in items]
    mlens = [it.msg_bytes for it in items]
    n = len(sizes)
    off, moff, p, q = [], [], 0, 0
    for c, m in zip(sizes, mlens):
        off.append(p)
        moff.append(q)
        p += (c + 255) // 256 * 256
        q += (m + 255) // 256 * 256
    covers = synth.uniform_bytes(p, synth.substream(synth.SEED_BASE + 4, 1), dev).cpu()
    covers = covers.pin_memory()
    msgs = synth.uniform_bytes(q, synth.substream(synth.SEED_BASE + 4, 2), dev).cpu()
    msgs = msgs.pin_memory()
    stego = torch.empty(p, dtype=torch.uint8).pin_memory()
    out = torch.zeros(q, dtype=torch.uint8).pin_memory()
    cv = [covers[o:o + c] for o, c in zip(off, sizes)]
    sv = [stego[o:o + c] for o, c in zip(off, sizes)]
    mv = [msgs[o:o + m] for o, m in zip(moff, mlens)]
    ov = [out[o:o + m] for o, m in zip(moff, mlens)]
    ej = S.Pipeline.jobs([dict(cover=cv[i], stego=sv[i], msg=mv[i], cover_bytes=sizes[i],
                               msg_bytes=mlens[i], flags=S.HEADER_BE32) for i in range(n)])
    xj = S.Pipeline.jobs([dict(cover=sv[i], msg=ov[i], cover_bytes=sizes[i],
                               msg_bytes=mlens[i], flags=S.HEADER_BE32) for i in range(n)])
    modes = {}
    for mode_name, mode in (("staged", S.PIPE_STAGED), ("auto", S.PIPE_AUTO)):
        te_, tx_ = tune if tune else ((0, 0, 0, 0), (0, 0, 0, 0))
        pipe = S.Pipeline(slots=slots, max_descs=4096, slot_bytes=slot_mb << 20, mode=mode,
                          tune_embed=te_, tune_extract=tx_)
        out.zero_()
        stego.zero_()
        pipe.embed(ej[:64], S.FUSE_STATS)  # warm-up
        pipe.extract(xj[:64])
        t_e, t_x = [], []
        for _ in range(3):
            t0 = time.perf_counter()
            re = pipe.embed(ej, S.FUSE_STATS, raw=True)
            t_e.append(time.perf_counter() - t0)
            t0 = time.perf_counter()
            rx = pipe.extract(xj, raw=True)
            t_x.append(time.perf_counter() - t0)
        pipe.close()
        re, rx = S.read_result(re), S.read_result(rx)
        assert all(r["status"] == 0 for r in re) and all(r["status"] == 0 for r in rx)
        assert all(rx[i]["msg_bytes"] == mlens[i] for i in range(n))
        assert all(torch.equal(ov[i], mv[i]) for i in range(n)), "host round trip differs"
        modes[mode_name] = (min(t_e), min(t_x))
    # the same batch with no staging at all: the batched kernels read and
    # write the pinned host arenas directly (zero copy)
    stream = torch.cuda.current_stream(dev)
    d_e = S.descs_to_device(S.pack_descs(
        [dict(cover=cv[i], stego=sv[i], msg=mv[i], cover_bytes=sizes[i], msg_bytes=mlens[i],
              flags=S.HEADER_BE32) for i in range(n)]), dev)
    d_x = S.descs_to_device(S.pack_descs(
        [dict(cover=sv[i], msg=ov[i], cover_bytes=sizes[i], msg_bytes=mlens[i],
              flags=S.HEADER_BE32) for i in range(n)]), dev)
    res_d = S.new_result(dev, n=n)
    ws = torch.empty(S.stego_batched_workspace_bytes(n), dtype=torch.uint8, device=dev)
    zc = {}
    for name, fn in (("embed", lambda: S.stego_embed_batched(d_e, n, res_d, S.FUSE_STATS, ws,
                                                             stream=stream)),
                     ("extract", lambda: S.stego_extract_batched(d_x, n, res_d, 0, ws,
                                                                 stream=stream))):
        fn()
        torch.cuda.synchronize(dev)
        ts = []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ts.append(e0.elapsed_time(e1) * 1e-3)
        zc[name + "_ms"] = round(min(ts) * 1e3, 2)
        zc[name + "_cover_gbs"] = round(sum(sizes) / min(ts) / 1e9, 1)
    assert all(torch.equal(ov[i], mv[i]) for i in range(n)), "zero-copy round trip differs"
    total = sum(sizes)
    msg_total = sum(mlens)
    carrying = sum(8 * (m + 4) for m in mlens)
    te, tx = modes["auto"]
    se, sx = modes["staged"]
    return {"workload": "4096 uneven covers (log-uniform sides 64..4096, 1 or 3 channels, "
                        "5-100% fill) in pinned host memory",
            "api": "stego_pipeline_embed / stego_pipeline_extract, %d slots of %d MiB, "
                   "up to 4096 covers per chunk, automatic mode (jobs without a read-back "
                   "are zero copy); best of 3, host wall clock" % (slots, slot_mb),
            "covers": n, "cover_bytes": total,
            "embed_ms": round(te * 1e3, 2), "extract_ms": round(tx * 1e3, 2),
            "embed_cover_gbs": round(total / te / 1e9, 1),
            "extract_cover_gbs": round(total / tx / 1e9, 1),
            "embed_link_bytes": {"h2d": total + msg_total, "d2h": total},
            "extract_link_bytes": {"h2d": carrying, "d2h": msg_total},
            "staged": {"what": "every job through the slots: covers and messages copied in, "
                               "stegos copied back by the copy engines",
                       "embed_ms": round(se * 1e3, 2), "extract_ms": round(sx * 1e3, 2),
                       "embed_cover_gbs": round(total / se / 1e9, 1),
                       "extract_cover_gbs": round(total / sx / 1e9, 1),
                       "embed_h2d_gbs": round((total + msg_total) / se / 1e9, 1),
                       "extract_h2d_gbs": round(total / sx / 1e9, 1)},
            "zero_copy_batched": dict(zc, api="stego_embed_batched / stego_extract_batched "
                                              "with descriptors pointing into the pinned host "
                                              "arenas (no staging copies); CUDA events")}


def run_e2e(args, S, torch, dev, stream, cover_d, msg_d, C, m):
    """Same step through the public API with pinned host buffers: host->device
    copy of the cover and message, embed, device->host copy of the stego and
    result; host->device copy of that stego, extract, device->host copy of
    the message and result."""
    cover_h = cover_d.cpu().pin_memory()
    msg_h = msg_d.cpu().pin_memory()
    stego_h = torch.empty(C, dtype=torch.uint8).pin_memory()
    out_h = torch.empty(m, dtype=torch.uint8).pin_memory()
    res_h = torch.empty(4, dtype=torch.int64).pin_memory()
    res2_h = torch.empty(4, dtype=torch.int64).pin_memory()
    c_d = torch.empty(C, dtype=torch.uint8, device=dev)
    m_d = torch.empty(m, dtype=torch.uint8, device=dev)
    s_d = torch.empty(C, dtype=torch.uint8, device=dev)
    x_d = torch.empty(C, dtype=torch.uint8, device=dev)
    o_d = torch.empty(m, dtype=torch.uint8, device=dev)
    r_d = S.new_result(dev)
    r2_d = S.new_result(dev)

    def step():
        c_d.copy_(cover_h, non_blocking=True)
        m_d.copy_(msg_h, non_blocking=True)
        S.stego_embed(c_d, s_d, m_d, S.HEADER_BE32 | S.FUSE_STATS, r_d, stream=stream)
        stego_h.copy_(s_d, non_blocking=True)
        res_h.copy_(r_d, non_blocking=True)
        x_d.copy_(stego_h, non_blocking=True)
        S.stego_extract(x_d, o_d, 0, S.HEADER_BE32, r2_d, stream=stream)
        out_h.copy_(o_d, non_blocking=True)
        res2_h.copy_(r2_d, non_blocking=True)

    for _ in range(2):
        step()
    torch.cuda.synchronize(dev)
    assert torch.equal(out_h, msg_h)
    n = args.e2e_steps
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(n):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / n
    return {"value": round(2.0 * C / (ms * 1e-3) / 1e9, 2), "unit": UNIT,
            "ms_per_step": round(ms, 4), "steps": n, "mode": "explicit copies",
            "h2d_bytes_per_step": 2 * C + m, "d2h_bytes_per_step": C + m + 64}


# ----------------------------------------------------------------------------
# CPU oracle (baseline leg and reference arm)
# ----------------------------------------------------------------------------

def oracle_round_trip(O, cover, msg, keep=None):
    """One embed + extract of (cover, msg) by the oracle; returns seconds.
    With `keep` (a dict), the stego and message it produced are stored."""
    import numpy as np
    out = np.empty_like(cover)
    t0 = time.perf_counter()
    st, _ = O.stream1_embed(cover, msg, header=True, out=out)
    st2, got = O.stream1_extract(out, cap=msg.size, header=True)
    dt = time.perf_counter() - t0
    assert st == 0 and st2 == 0 and got.size == msg.size
    if keep is not None:
        keep["stego"], keep["msg"] = out, got
    return dt


def host_cpu() -> str:
    """Model name of the host CPU (lscpu, else /proc/cpuinfo) and core count."""
    name = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                name = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not name:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu model")):
                        name = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return "%s, %d cores" % (name or "unknown CPU", os.cpu_count() or 0)


def run_cpu_baseline(cover, msg, budget_s=12.0, gpu_stego=None, gpu_msg=None):
    """The oracle's round trips on one host core.  With the GPU's stego and
    extracted message of the timed configuration, the last round trip's
    outputs are compared with them byte for byte (`matches_gpu`)."""
    import numpy as np
    import oracle
    O = oracle.load()
    times, keep = [], {}
    while (sum(times) < budget_s or len(times) < 5) and len(times) < 50:
        times.append(oracle_round_trip(O, cover, msg, keep))
    med = statistics.median(times)
    out = {"value": round(2.0 * cover.size / med / 1e9, 4), "unit": UNIT,
           "cores": 1, "kind": "oracle", "host": host_cpu(),
           "sample": "median of %d embed+extract round trips of the whole %d-byte cover "
                     "(single-threaded C oracle, %.1f s)" % (len(times), cover.size, sum(times))}
    if gpu_stego is not None:
        out["matches_gpu"] = bool(np.array_equal(keep["stego"], gpu_stego) and
                                  np.array_equal(keep["msg"], gpu_msg))
    return out


def run_cpu_all_cores(cover, msg, budget_s=6.0):
    """The same oracle on every host core: the cover is cut into one
    independent cover per core (16-byte multiples), each carrying its own
    full-capacity message, and the round trips run in parallel threads (the
    oracle's C calls release the GIL)."""
    from concurrent.futures import ThreadPoolExecutor
    import oracle
    O = oracle.load()
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    part = cover.size // cores // 16 * 16
    jobs = [(cover[i * part:(i + 1) * part], msg[:part // 8 - 4]) for i in range(cores)]
    times = []
    with ThreadPoolExecutor(cores) as ex:
        while (sum(times) < budget_s or len(times) < 5) and len(times) < 50:
            t0 = time.perf_counter()
            list(ex.map(lambda j: oracle_round_trip(O, j[0], j[1]), jobs))
            times.append(time.perf_counter() - t0)
    med = statistics.median(times)
    return {"value": round(2.0 * part * cores / med / 1e9, 4), "unit": UNIT,
            "cores": cores, "kind": "oracle",
            "sample": "median of %d rounds of %d parallel embed+extract round trips, one "
                      "independent %d-byte cover per core cut from the same cover (%.1f s)"
                      % (len(times), cores, part, sum(times))}


def run_reference(args, rank, world):
    """The CPU oracle as the reference arm: each step one embed + extract of
    the workload's whole cover, or of a prefix of it when the whole cover
    would not let all steps finish in about a minute (`config.workload` and
    `sample_bytes` say which)."""
    if rank != 0:
        return None
    import numpy as np
    import oracle
    from paper_0912_0947_gb300 import synth
    O = oracle.load()
    w = synth.single_8192()
    # the same bytes as the GPU arm's cover/message, generated on the host
    C_full = w.cover_bytes
    # calibrate on 8 MiB
    calib = 8 << 20
    cov = synth.uniform_bytes_np(calib, synth.substream(w.seed, 1))
    msg = synth.uniform_bytes_np(calib // 8 - 4, synth.substream(w.seed, 2))
    rate = calib / oracle_round_trip(O, cov, msg)  # cover bytes / s
    total_steps = args.steps + args.warmup
    sample = int(min(C_full, max(1 << 16, rate * args.ref_seconds / total_steps)))
    sample -= sample % 16
    cov = synth.uniform_bytes_np(sample, synth.substream(w.seed, 1))
    msg = synth.uniform_bytes_np(sample // 8 - 4, synth.substream(w.seed, 2))
    for _ in range(args.warmup):
        oracle_round_trip(O, cov, msg)
    t = sum(oracle_round_trip(O, cov, msg) for _ in range(args.steps))
    value = 2.0 * sample * args.steps / t / 1e9
    whole = sample == C_full - C_full % 16
    desc = ("the whole %d-byte 8192x8192x3 cover with a %d-byte message (full capacity) "
            "per step" % (sample, sample // 8 - 4)) if whole else \
           ("prefix of %d bytes of the 8192x8192x3 cover with a %d-byte message "
            "(full capacity of the prefix) per step" % (sample, sample // 8 - 4))
    return {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(t / args.steps * 1e3, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": "single 8192x8192x3 uint8 cover, full 1-bit capacity; "
                               "embed + extract (CPU oracle, %s)" % (
                                   "whole cover" if whole else "bounded prefix"),
                   "cover_bytes": C_full, "sample_bytes": sample},
        "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--steady-pairs", type=int, default=6,
                    help="distinct cover/stego sets of the steady-state leg (0: skip)")
    ap.add_argument("--steady-only", action="store_true",
                    help="run only the steady-state sequence (for an ncu capture)")
    ap.add_argument("--profile-case", default="",
                    help="co,so,mo: run only two embed + extract calls of the 201 MB cover "
                         "at those byte offsets (for an ncu capture)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-seconds", type=float, default=60.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--shape-embed", default="",
                    help="fixed launch shape threads,vec,ctas_per_sm,tile_bytes for the embed "
                         "(tile_bytes > 0: shared-memory staged kernel with that ring)")
    ap.add_argument("--shape-extract", default="", help="same for the extract")
    ap.add_argument("--serving-seconds", type=float, default=20.0,
                    help="arrival span per rate of the serving leg")
    ap.add_argument("--serving-max-requests", type=int, default=1000000,
                    help="request cap per rate of the serving leg")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--uneven-count", type=int, default=0,
                    help="covers in the uneven batched leg (default 4096)")
    ap.add_argument("--video-frames", type=int, default=0,
                    help="frames in the video batched leg (default 600)")
    ap.add_argument("--legs", default="",
                    help="comma list of extra legs: batched_uneven,batched_video,"
                         "batched_video_paper2,paper2,streamk,serving,small,extract_gather,"
                         "batched_uneven_host,batched_uneven_misaligned,single_misaligned,"
                         "split_cover, "
                         "or none "
                         "(default: all with one GPU, none with several)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if line is not None:
            print(json.dumps(line), flush=True)
        return 0

    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    line = run_ours(args, rank, world, local_rank)
    if line is not None:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
