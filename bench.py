#!/usr/bin/env python3
"""Benchmark of the per-thread stream generation and its Ising consumer.

Default (N=1): the bulk workload -- 2^20 resident instances of every
generator kind, 1024 draws each (2^30 outputs per call; the block-shared
MT19937 and lagged Fibonacci generators as 32768 warp-shared generators x
2^15 draws), written to HBM as u32, exact
uniform f32 and Box-Muller normals, and consumed in registers (u32 XOR
reduce).  One step = those 40 calls (ten kinds x four forms).  `value` = outputs of all ranks /
device time (Gnum/s).  Extra keys report the Ising sweep (flips/ns) and
the other workloads.

`--case gen|ising|all` runs one kernel configuration on a small case for a
profiler instead (see run_case).

Under torchrun (N>1) each rank holds its own shard of an N x 2^20-instance
generator (global instance indices, no collective on the data path):
weak scaling.

`--impl reference` times the CPU oracle (the reference implementation of
the method for this build) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RNG Gnum/s (frac of HBM peak); Ising flips/ns; served p50/p99 vs plain"
N_INST = 1 << 20
K_DRAWS = 1024
MT_GENS = 1 << 15   # one generator per warp: 2^20 threads
MT_DRAWS = 1 << 15
SEED = 0x0123456789ABCDEF
FORMS = ["u32", "f32", "normal", "u32_xor"]
# state bytes moved per instance and call: load + store of the state, plus
# the MWC multiplier read; Philox only reads its key (the position is the
# handle's counter)
STATE_TRAFFIC = {0: 8, 1: 16, 2: 20, 3: 48, 4: 8, 5: 8, 6: 2 * 624 * 4, 7: 8, 8: 2 * 521 * 4, 9: 2 * 1279 * 4}
# LCG32, LCG64, MWC, XORWOW, Philox4x32-10, XS1024W, MT19937, Philox4x32-7,
# lagged Fibonacci (521, 353) and (1279, 861)
# Algorithmic integer operations per number of each generator's recurrence
# (the roof of the consume-in-register form, which writes 4 B per instance):
# LCG32 one multiply-add; LCG64 a 64-bit multiply-add (3 32-bit operations);
# MWC a 32 x 32 -> 64-bit multiply-add and a move; XORWOW four shifts, four
# XORs (two three-input), the Weyl add and the output add (8); Philox4x32-10
# per 4 numbers 10 rounds of two wide multiplies, three XORs and two key adds
# (18 per number; 7 rounds: 12.6); the 1024-bit generator per word three
# funnel shifts, three XORs, the three pairs of neighbour words (6 shuffles)
# and the Weyl output (16); MT19937 per word the twist (mask merge, shift,
# conditional XOR, XOR: 4) and the tempering (4 shifts, 4 masked XORs: 8);
# lagged Fibonacci one add.
ALG_OPS = {0: 1.0, 1: 3.0, 2: 2.0, 3: 8.0, 4: 18.0, 5: 16.0, 6: 12.0, 7: 12.6, 8: 1.0, 9: 1.0}
N_KINDS = 10
SHARED = (6, 8, 9)  # block-shared kinds: one state per warp, 2^15 generators x 2^15 draws


def shard_range(rank: int, world: int, per_rank: int):
    """Instances [first, first + count) of an (world * per_rank)-instance
    generator held by `rank` (weak scaling: per-rank work is fixed)."""
    return rank * per_rank, per_rank, world * per_rank


def max_over_ranks(value: float, dist, device=None) -> float:
    """The slowest rank's time: every rank contributes its elapsed time."""
    import torch
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured", "sm_max_mhz": d.get("sm_max_mhz")}
    return {"hbm_gbs": 6800.0, "source": "fallback", "sm_max_mhz": 2070.0}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-i",
                 str(self.device), "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sms, maxs, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sms.append(float(parts[0]))
                maxs.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sms:
            return None
        return {"sm_mhz": statistics.median(sms), "sm_max_mhz": max(maxs), "samples": len(sms),
                "reasons": sorted(reasons)}


def file_hash(paths):
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


GEN_SOURCES = ["paper_1204_6193_gb300/csrc/gen.cu", "paper_1204_6193_gb300/csrc/gen_device.cuh",
               "paper_1204_6193_gb300/csrc/lfib.cu", "paper_1204_6193_gb300/csrc/normal_tables.h"]


def _ncu_summary():
    """The committed ncu summary of the generation kernels, if their sources
    are unchanged since it was captured."""
    p = os.path.join(ROOT, "profiles", "gen_bulk_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    return d if d.get("source_hash") == file_hash(GEN_SOURCES) else None


def roof_of(form: str, hbm: dict, alg: dict) -> dict:
    """The roof of a generation call by the algorithmic work it must do: a
    call that writes its numbers is bound by HBM (output bytes plus the
    state's load and store); the consume-in-register call writes 4 bytes per
    instance and is bound by the integer operations of the recurrence
    (ALG_OPS) against the instruction-issue roof."""
    if form == "u32_xor":
        return {"bound": "alu", **alg}
    return {"bound": "hbm", **hbm}


def ncu_traffic(kernel_key: str):
    """DRAM bytes per launch (ncu), scaled to the bench's launch."""
    d = _ncu_summary()
    v = d.get("traffic_bytes_per_launch", {}).get(kernel_key) if d else None
    return float(v) if v is not None else None


def ncu_inst_per_output(kernel_key: str):
    """Thread instructions executed per output (ncu smsp__thread_inst_executed)."""
    d = _ncu_summary()
    v = d.get("thread_inst_per_output", {}).get(kernel_key) if d else None
    return float(v) if v is not None else None


def bulk_config(world: int) -> dict:
    """The bulk workload, as both arms name it."""
    return {
        "workload": "bulk generation: 2^20 resident instances x 1024 draws per call (MT19937 and the "
                    "lagged Fibonacci (521, 353), (1279, 861): 32768 warp-shared generators x 2^15), "
                    "10 generators x {u32, f32, normal} written to HBM + u32 consumed in registers "
                    "(XOR reduce); 40 calls per step",
        "instances_per_gpu": N_INST, "draws_per_call": K_DRAWS,
        "outputs_per_step_per_gpu": N_KINDS * len(FORMS) * N_INST * K_DRAWS,
        "layout": "step-major (block-shared kinds: instance-major)",
        "l2": "no flush: every write call streams 4 GiB (> 129 MB L2)", "seed": hex(SEED),
        "parallelism": f"instance shards x{world}",
    }


# ------------------------------------------------------------------ GPU arm
class Bulk:
    def __init__(self, R, torch, rank, world):
        self.R, self.torch = R, torch
        self.handles = {}
        for kind in range(N_KINDS):
            per = MT_GENS if kind in SHARED else N_INST
            first, n, total = shard_range(rank, world, per)
            h = R.rng_create_shard(kind, total, first, n, 0)
            R.rng_seed(h, SEED)
            self.handles[kind] = (h, n)
        self.out = torch.empty(N_INST * K_DRAWS, dtype=torch.int32, device="cuda")
        self.red = torch.empty(N_INST, dtype=torch.int32, device="cuda")

    def calls(self):
        """(name, kind, form, fn, n, K, layout) for one step."""
        R = self.R
        res = []
        for kind in range(N_KINDS):
            h, n = self.handles[kind]
            K = MT_DRAWS if kind in SHARED else K_DRAWS
            lay = R.RNG_INSTANCE_MAJOR if kind in SHARED else R.RNG_STEP_MAJOR
            for form in FORMS:
                res.append((f"{R.KIND_NAMES[kind]}/{form}", kind, form, h, n, K, lay))
        return res

    def launch(self, c, stream):
        R = self.R
        _, kind, form, h, n, K, lay = c
        if form == "u32":
            R.rng_generate_u32(h, self.out.data_ptr(), K, lay, stream)
        elif form == "f32":
            R.rng_generate_f32(h, self.out.data_ptr(), K, lay, stream)
        elif form == "normal":
            R.rng_generate_normal(h, self.out.data_ptr(), K, lay, stream)
        else:
            R.rng_generate_u32(h, self.red.data_ptr(), K, R.RNG_XOR_REDUCE, stream)

    def algorithmic_bytes(self, c):
        _, kind, form, h, n, K, lay = c
        out = n * 4 if form == "u32_xor" else n * K * 4
        return out + STATE_TRAFFIC[kind] * n

    def close(self):
        for h, _ in self.handles.values():
            self.R.rng_destroy(h)


def run_gpu(args):
    import torch
    import torch.distributed as dist

    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_1204_6193_gb300 as R

    peaks = load_peaks()
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    # pipe throughputs of this GPU, measured outside the timed region
    issue_peaks = R.rng_issue_peaks(sptr)
    bulk = Bulk(R, torch, rank, world)
    calls = bulk.calls()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        for c in calls:
            bulk.launch(c, sptr)
    barrier()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)  # let the sampler start before the timed region
    barrier()
    ev = []
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        for c in calls:
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            bulk.launch(c, sptr)
            b.record(stream)
            ev.append((c, a, b))
    t1.record(stream)
    barrier()
    clk = clocks.stop()
    elapsed_ms = max_over_ranks(t0.elapsed_time(t1), dist if world > 1 else None, "cuda")

    per = {}
    for c, a, b in ev:
        d = per.setdefault(c[0], {"ms": [], "call": c})
        d["ms"].append(a.elapsed_time(b))
    outputs_per_step_rank = sum((c[4] * c[5]) for c in calls)
    total_outputs = outputs_per_step_rank * world * args.steps
    value = total_outputs / (elapsed_ms * 1e-3) / 1e9

    # instruction-issue roof: one warp instruction per scheduler and cycle,
    # 4 schedulers per SM, at the highest SM clock sampled during the timed
    # region (the measured FFMA rate of rng_issue_peaks when no clock was read)
    n_sms = torch.cuda.get_device_properties(local).multi_processor_count
    if clk and clk.get("sm_max_mhz"):
        issue_peak = n_sms * 4 * 32 * clk["sm_max_mhz"] * 1e6 / 1e12
        issue_src = f"{n_sms} SMs x 4 schedulers x 32 threads x {clk['sm_max_mhz']:.0f} MHz (one warp instruction " \
                    "per scheduler and cycle)"
    elif issue_peaks:
        issue_peak = issue_peaks["ffma"] / 1e12
        issue_src = "measured FFMA rate (rng_issue_peaks)"
    else:
        issue_peak, issue_src = None, None

    def issue_of(name, c, avg_ms):
        """Executed thread instructions (ncu count per output) against the
        issue roof: why a kernel sits where it does, not its roofline."""
        ipo = ncu_inst_per_output(name)
        if ipo is None or issue_peak is None:
            return None
        ach = ipo * c[4] * c[5] / (avg_ms * 1e-3) / 1e12
        return {"inst_per_output": round(ipo, 2), "achieved_tinst_s": round(ach, 2),
                "peak_tinst_s": round(issue_peak, 2), "frac": round(ach / issue_peak, 3), "peak_source": issue_src,
                "source": "executed thread instructions per output (profiles/gen_bulk_traffic.json, ncu) x "
                          "outputs / CUDA-event time"}

    def hbm_of(c, avg_ms):
        ach = bulk.algorithmic_bytes(c) / (avg_ms * 1e-3) / 1e9
        return {"achieved": round(ach, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": round(ach / peaks["hbm_gbs"], 4),
                "peak_source": f"{peaks['source']} (MEASURED_PEAKS.json hbm_gbs, copy bandwidth)"
                if peaks["source"] == "measured" else "fallback 6.8 TB/s",
                "algorithmic_bytes_per_launch": bulk.algorithmic_bytes(c)}

    def alg_of(c, avg_ms):
        ops = ALG_OPS[c[1]]
        ach = ops * c[4] * c[5] / (avg_ms * 1e-3) / 1e12
        return {"achieved": round(ach, 2), "peak": round(issue_peak, 2) if issue_peak else None,
                "unit": "T integer ops/s", "frac": round(ach / issue_peak, 4) if issue_peak else None,
                "peak_source": issue_src, "ops_per_number": ops}

    detail = {}
    best = None
    for name, d in per.items():
        c = d["call"]
        avg = sum(d["ms"]) / len(d["ms"])
        tot = sum(d["ms"])
        rec = {"ms": round(avg, 4), "gnum_s": round(c[4] * c[5] / (avg * 1e-3) / 1e9, 1)}
        if c[2] == "u32_xor":
            a = alg_of(c, avg)
            rec.update({"bound": "alu", "frac_alg_ops": a["frac"], "ops_per_number": a["ops_per_number"]})
        else:
            h_ = hbm_of(c, avg)
            rec.update({"bound": "hbm", "gb_s": h_["achieved"], "frac_hbm": h_["frac"]})
        iss = issue_of(name, c, avg)
        if iss:
            rec["issue_frac"] = iss["frac"]
            rec["inst_per_output"] = iss["inst_per_output"]
        detail[name] = rec
        if best is None or tot > best[1]:
            best = (name, tot, avg, c)
    name, tot, avg, c = best
    step_ms_total = sum(sum(d["ms"]) for d in per.values())
    roofline = {"kernel": name, **roof_of(c[2], hbm_of(c, avg), alg_of(c, avg))}
    roofline.update({
        "share_of_step": round(tot / step_ms_total, 3),
        "launch_ms": round(avg, 4),
        "timing": "mean CUDA-event time of the kernel's launches inside the timed region, on its stream",
        "traffic": ncu_traffic(name),
        "traffic_source": "dram__bytes_read.sum + dram__bytes_write.sum per launch (profiles/gen_bulk_traffic.json)",
        "issue": issue_of(name, c, avg),
    })

    # end to end through the C ABI with host buffers: each step reseeds from a
    # host seed and every output ends in pinned host memory, either written
    # there directly by the kernels (host memory is device-addressable over
    # NVLink-C2C) or generated into device memory and copied on a second
    # stream while the next call generates; the faster is reported
    e2e = None
    if not args.no_e2e:
        e_steps = max(1, min(2, args.steps))
        host = torch.empty(N_INST * K_DRAWS, dtype=torch.int32, pin_memory=True)
        hred = torch.empty(N_INST, dtype=torch.int32, pin_memory=True)
        out_bytes = [c[4] * 4 if c[2] == "u32_xor" else c[4] * c[5] * 4 for c in calls]

        def run_direct():
            for st in range(e_steps):
                for kind in range(N_KINDS):
                    R.rng_seed(bulk.handles[kind][0], SEED + 1 + st)
                for c in calls:
                    launch_into(c, hred.data_ptr() if c[2] == "u32_xor" else host.data_ptr())

        def launch_into(c, ptr):
            _, kind, form, h, n, K, lay = c
            if form == "u32":
                R.rng_generate_u32(h, ptr, K, lay, sptr)
            elif form == "f32":
                R.rng_generate_f32(h, ptr, K, lay, sptr)
            elif form == "normal":
                R.rng_generate_normal(h, ptr, K, lay, sptr)
            else:
                R.rng_generate_u32(h, ptr, K, R.RNG_XOR_REDUCE, sptr)

        copy_stream = torch.cuda.Stream()
        dev2 = torch.empty(N_INST * K_DRAWS, dtype=torch.int32, device="cuda")
        bufs = [bulk.out, dev2]
        done_ev = [torch.cuda.Event(), torch.cuda.Event()]

        def run_copy():
            i = 0
            for st in range(e_steps):
                for kind in range(N_KINDS):
                    R.rng_seed(bulk.handles[kind][0], SEED + 1 + st)
                for c in calls:
                    b = bufs[i % 2]
                    stream.wait_event(done_ev[i % 2])  # copy from two calls ago has drained
                    src = bulk.red if c[2] == "u32_xor" else b
                    launch_into(c, src.data_ptr())
                    gen_ev = torch.cuda.Event()
                    gen_ev.record(stream)
                    copy_stream.wait_event(gen_ev)
                    nb = out_bytes[calls.index(c)] // 4
                    with torch.cuda.stream(copy_stream):
                        (hred if c[2] == "u32_xor" else host)[:nb].copy_(src[:nb], non_blocking=True)
                    done_ev[i % 2].record(copy_stream)
                    i += 1
            stream.wait_stream(copy_stream)

        variants, step_ms = {}, {}
        for name, fn in (("direct", run_direct), ("copy_overlapped", run_copy)):
            barrier()
            s0 = torch.cuda.Event(enable_timing=True)
            s1 = torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            fn()
            s1.record(stream)
            barrier()
            e_ms = max_over_ranks(s0.elapsed_time(s1), dist if world > 1 else None, "cuda")
            variants[name] = round(outputs_per_step_rank * world * e_steps / (e_ms * 1e-3) / 1e9, 2)
            step_ms[name] = e_ms / e_steps
        best = max(variants, key=variants.get)
        # the host link's own roof: a plain pinned device-to-host copy of the
        # 4 GiB output buffer, best of three, CUDA events on this stream
        link = []
        for _ in range(3):
            c0 = torch.cuda.Event(enable_timing=True)
            c1 = torch.cuda.Event(enable_timing=True)
            c0.record(stream)
            host.copy_(bulk.out, non_blocking=True)
            c1.record(stream)
            torch.cuda.synchronize()
            link.append(host.numel() * 4 / (c0.elapsed_time(c1) * 1e-3) / 1e9)
        link_gbs = max(link)
        d2h = sum(out_bytes)
        achieved_gbs = d2h / (step_ms[best] * 1e-3) / 1e9
        e2e = {"value": variants[best], "unit": "Gnum/s", "h2d_bytes_per_step": 0,
               "d2h_bytes_per_step": d2h, "steps": e_steps, "variant": best, "variants": variants,
               "roofline": {"bound": "host link", "achieved": round(achieved_gbs, 1), "peak": round(link_gbs, 1),
                            "unit": "GB/s", "frac": round(achieved_gbs / link_gbs, 3),
                            "peak_source": "pinned device-to-host copy of 4 GiB (torch copy_, best of 3, CUDA "
                                           "events), measured in this run"},
               "note": "seed passed by value (no input arrays); every output lands in pinned host memory"}
        del dev2

    bulk.close()
    extra = {}
    if rank == 0 and not args.no_ising:
        extra["ising"] = ising_section(R, torch, args)
    if rank == 0 and not args.no_batch:
        extra["batched"] = batch_section(R, torch, args)
    if rank == 0 and not args.no_serve:
        extra["served"] = serve_section(R, torch, args)

    line = None
    if rank == 0:
        cpu = None if (args.no_cpu or world > 1) else cpu_baseline(args)
        line = {
            "metric": METRIC,
            "value": round(value, 2),
            "unit": "Gnum/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": round(elapsed_ms / args.steps, 3),
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "u32",
            "data": "synthetic",
            "config": bulk_config(world),
            "roofline": roofline,
            "issue_peaks": {k: round(v / 1e12, 2) for k, v in issue_peaks.items()} | {
                "unit": "T thread-instructions/s (whole GPU)", "source": "rng_issue_peaks microbenchmark"},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clk,
            "gpu_launches": len(ev),
            "detail": detail,
        }
        line.update(extra)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return line


# ------------------------------------------------------------ Ising (config 3)
BETA_C = 0.44068679350977151


# (kind, flags) of the Ising consumers: the paper's generator, xorwow, both
# Philox variants (Philox4x32-7 with intrinsic keys, Sec. 7) and LCG32
ISING_KINDS = ((5, 0), (3, 0), (4, 0), (7, 8), (0, 0))


def _ising_kind_name(R, kind, flags):
    return R.KIND_NAMES[kind] + ("_intrinsic" if flags & R.RNG_PHILOX_INTRINSIC_KEY else "")


def _time_sweeps(R, torch, h, n, plain=False):
    stream = torch.cuda.current_stream()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    (R.ising_sweep_plain if plain else R.ising_sweep)(h, n, 0, stream.cuda_stream)
    b.record(stream)
    torch.cuda.synchronize()
    R.ising_observables(h)  # surfaces a timed-out wait, if any
    return a.elapsed_time(b)


def ising_section(R, torch, args):
    """flips/ns = L^2 sweeps / device time, persistent fused kernel vs one
    launch per half-sweep, at beta_c with G = 2 and a random start."""
    out = {"beta": BETA_C, "G": 2, "unit": "flips/ns"}
    n = args.ising_sweeps
    for L in (1024, 64):
        for layout, lname in ((R.ISING_INT8, "int8"), (R.ISING_MULTISPIN32, "multispin32")):
            for kind, flags in ISING_KINDS:
                if L == 64 and kind not in (R.RNG_XS1024W, R.RNG_XORWOW):
                    continue
                h = R.ising_create(L, BETA_C, layout, kind, flags, SEED, 2)
                try:
                    tuned = R.ising_autotune(h, 64)
                    R.ising_sweep(h, 50)
                    ms = _time_sweeps(R, torch, h, n)
                    nplain = max(20, n // 10)
                    ms_plain = _time_sweeps(R, torch, h, nplain, plain=True)
                    key = f"L{L}/{lname}/{_ising_kind_name(R, kind, flags)}"
                    by_depth = {}
                    if L == 1024:
                        # both exchange variants in the one-strip-per-SM shape:
                        # after every half-sweep (1), once per sweep with the
                        # two-row halo (2)
                        launch, depth = R.ising_get_launch(h), R.ising_get_halo_depth(h)
                        R.ising_set_launch(h, 1024, 1, 0)
                        for d in (1, 2):
                            R.ising_set_halo_depth(h, d)
                            R.ising_sweep(h, 50)
                            by_depth[f"depth{d}"] = round(L * L * n / (_time_sweeps(R, torch, h, n) * 1e6), 2)
                        R.ising_set_launch(h, launch["threads"], launch["ctas_per_sm"], launch["min_sites"])
                        R.ising_set_halo_depth(h, depth)
                    out[key] = {
                        "flips_per_ns": round(L * L * n / (ms * 1e6), 2),
                        "us_per_sweep": round(1e3 * ms / n, 3),
                        "plain_flips_per_ns": round(L * L * nplain / (ms_plain * 1e6), 3),
                        "sweeps_timed": n, "launch": tuned, "halo_depth": R.ising_get_halo_depth(h),
                        **({"flips_per_ns_by_halo_depth": by_depth} if by_depth else {}),
                        "plan": R.ising_plan_info(h),
                    }
                finally:
                    R.ising_destroy(h)
    # the block-shared generators (MT19937, lagged Fibonacci; Table 1's
    # Fibonacci rows): one generator per 32 streams, states streamed through
    # L2 every half-sweep (the per-half-sweep path)
    n_sh = max(20, n // 50)
    for L in (1024, 64):
        for layout, lname in ((R.ISING_INT8, "int8"), (R.ISING_MULTISPIN32, "multispin32")):
            for kind in (R.RNG_MT19937_SHARED, R.RNG_LFIB521, R.RNG_LFIB1279):
                if L == 64 and layout != R.ISING_INT8:
                    continue
                h = R.ising_create(L, BETA_C, layout, kind, 0, SEED, 2)
                try:
                    R.ising_sweep(h, 5)
                    ms = _time_sweeps(R, torch, h, n_sh)
                    out[f"L{L}/{lname}/{R.KIND_NAMES[kind]}"] = {
                        "flips_per_ns": round(L * L * n_sh / (ms * 1e6), 3), "us_per_sweep": round(1e3 * ms / n_sh, 2),
                        "sweeps_timed": n_sh, "path": "per half-sweep: generators write 32 G words each to an "
                                                      "L2-resident buffer, one kernel consumes them"}
                finally:
                    R.ising_destroy(h)
    out["multihit"] = multihit_section(R, torch, n)
    if not args.no_cpu:
        out["cpu_oracle"] = ising_oracle_rate()
    return out


def ising_oracle_rate(sweeps: int = 20):
    """The CPU oracle's checkerboard sweep of the 1024^2 lattice at beta_c
    (xorwow, G = 2), single-threaded: flips/ns beside the GPU's."""
    import oracle as O
    O.ising_run(64, BETA_C, 3, SEED, 2)  # loads the oracle
    t0 = time.perf_counter()
    O.ising_run(1024, BETA_C, 3, SEED, sweeps)
    dt = time.perf_counter() - t0
    return {"flips_per_ns": round(1024 * 1024 * sweeps / (dt * 1e9), 4), "cores": 1,
            "sample": f"{sweeps} sweeps of L=1024 int8, xorwow, {dt:.2f} s"}


def _time_rounds(R, torch, h, rounds, k, strips):
    stream = torch.cuda.current_stream()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    R.ising_sweep_multihit(h, rounds, k, strips, 0, stream.cuda_stream)
    b.record(stream)
    torch.cuda.synchronize()
    R.ising_observables(h)
    return a.elapsed_time(b)


def multihit_section(R, torch, n):
    """Multi-hit (double checkerboard) rounds: k sweeps per strip phase, k = 1,
    2 (Sec. 7) and 100 (the t_up^{k=100} column of Table 1), flips/ns = L^2 k
    rounds / device time; the strip count is the fastest of a few on a short
    probe."""
    out = {}
    for L, cands in ((1024, (256, 512, 1024)), (64, (2, 4, 8, 16))):
        for layout, lname in ((R.ISING_INT8, "int8"), (R.ISING_MULTISPIN32, "multispin32")):
            for kind, flags in ISING_KINDS:
                if L == 64 and kind not in (R.RNG_XS1024W, R.RNG_XORWOW):
                    continue
                h = R.ising_create(L, BETA_C, layout, kind, flags, SEED, 2)
                try:
                    best = None
                    for strips in cands:
                        try:
                            R.ising_sweep_multihit(h, 1, 100, strips)
                            ms = _time_rounds(R, torch, h, 2, 100, strips)
                        except R.RngError:
                            continue
                        if best is None or ms < best[0]:
                            best = (ms, strips)
                    if best is None:
                        continue
                    strips = best[1]
                    rec = {"strips": strips}
                    for k in (1, 2, 100):
                        rounds = max(2, n // k)
                        ms = _time_rounds(R, torch, h, rounds, k, strips)
                        rec[f"k{k}_flips_per_ns"] = round(L * L * k * rounds / (ms * 1e6), 2)
                        rec[f"k{k}_rounds_timed"] = rounds
                    out[f"L{L}/{lname}/{_ising_kind_name(R, kind, flags)}"] = rec
                finally:
                    R.ising_destroy(h)
    return out


# --------------------------------------------------------- batched (config 4)
def batch_workload(n=256, seed=7):
    import numpy as np
    rng = np.random.default_rng(seed)
    Ls = (2 ** rng.integers(4, 10, n)).tolist()  # 16 .. 512, uniform over exponents
    betas = rng.uniform(0.30, 0.60, n).tolist()
    kinds = [3 if b % 2 == 0 else 5 for b in range(n)]  # xorwow / the paper's generator
    return Ls, betas, kinds


def batch_section(R, torch, args):
    Ls, betas, kinds = batch_workload()
    sites = sum(L * L for L in Ls)
    n = args.batch_sweeps
    h = R.ising_batch_create(Ls, betas, kinds, SEED, 2)
    try:
        tuned = R.ising_autotune(h, 32)
        R.ising_batch_sweep(h, n)  # captures the graph; also warm-up
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        R.ising_batch_sweep(h, n, 0, stream.cuda_stream)  # graph replay
        b.record(stream)
        torch.cuda.synchronize()
        R.ising_batch_observables(h, 0)
        ms = a.elapsed_time(b)
        plan = R.ising_plan_info(h)
    finally:
        R.ising_destroy(h)
    # one launch per lattice: each lattice alone through ising_sweep
    nb = max(10, n // 10)
    hs = [R.ising_create(L, bt, 0, k, 0, int(O_seed_word(SEED, i)), 2) for i, (L, bt, k) in
          enumerate(zip(Ls, betas, kinds))]
    try:
        for hh in hs:
            R.ising_sweep(hh, 2)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        stream = torch.cuda.current_stream()
        a.record(stream)
        for hh in hs:
            R.ising_sweep(hh, nb, 0, stream.cuda_stream)
        b.record(stream)
        torch.cuda.synchronize()
        ms_alone = a.elapsed_time(b)
    finally:
        for hh in hs:
            R.ising_destroy(hh)
    fl = sites * n / (ms * 1e6)
    fl_alone = sites * nb / (ms_alone * 1e6)
    return {"lattices": len(Ls), "sites": sites, "sweeps": n, "ms": round(ms, 2), "flips_per_ns": round(fl, 2),
            "one_launch_per_lattice": {"sweeps": nb, "ms": round(ms_alone, 2), "flips_per_ns": round(fl_alone, 3)},
            "speedup": round(fl / fl_alone, 2), "launch": tuned, "plan": plan,
            "workload": "L log-uniform over {16..512}, beta U[0.30,0.60], xorwow/xs1024w alternating, G=2, "
                        "per generator kind, waves of lattices whose streams fit the registers (one persistent launch each per " \
                        "4096 sweeps), all replayed from one CUDA graph"}


def O_seed_word(seed, k):
    """SplitMix64 word w_k of the master seed (the batch seeds lattice b
    with w_b); computed here only to build the one-lattice-per-launch
    baseline with the same seeds."""
    m = (1 << 64) - 1
    z = (seed + (k + 1) * 0x9E3779B97F4A7C15) & m
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
    return z ^ (z >> 31)


# ---------------------------------------------------------- served (config 5)
def serve_requests(R, n, seed=3):
    import numpy as np
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        r = R.rng_request_t()
        if rng.random() < 0.8:
            r.type = R.RNG_REQ_DRAW
            r.kind = int(rng.integers(0, 6))
            r.out = int(rng.integers(0, 3))
            r.count = int(2 ** rng.uniform(10, 26)) // 2 * 2
            r.seed = int(rng.integers(0, 64))
            r.offset = int(rng.integers(0, 4096)) << 20
        else:
            r.type = R.RNG_REQ_SWEEP
            r.kind = int(rng.choice([3, 5]))
            r.L = int(rng.choice([64, 128, 256, 512, 1024]))
            r.beta = float(rng.uniform(0.3, 0.6))
            r.sweeps = int(10 ** rng.uniform(1, 3))
            r.seed = int(rng.integers(0, 1 << 62))
        reqs.append(r)
    return reqs


def _serve_run(R, srv, reqs, rate):
    """Submits reqs with Poisson arrivals at `rate` per second (rate None: all
    at once); returns (latencies in ms, wall seconds)."""
    import threading
    import numpy as np
    rng = np.random.default_rng(1)
    gaps = rng.exponential(1.0 / rate, len(reqs)) if rate else np.zeros(len(reqs))
    tickets = [None] * len(reqs)
    lat = [None] * len(reqs)
    wait = [None] * len(reqs)
    ready = threading.Semaphore(0)

    def collector():
        for i in range(len(reqs)):
            ready.acquire()
            res = R.rng_server_wait(srv, tickets[i], 600.0)
            lat[i] = (res.t_done_ns - res.t_submit_ns) / 1e6
            wait[i] = (res.t_start_ns - res.t_submit_ns) / 1e6
            R.rng_server_fetch(srv, tickets[i], None, 0)

    th = threading.Thread(target=collector)
    th.start()
    t0 = time.perf_counter()
    due = t0
    for i, r in enumerate(reqs):
        due += gaps[i]
        while True:
            now = time.perf_counter()
            if now >= due:
                break
            time.sleep(min(due - now, 0.0005))
        tickets[i] = R.rng_server_submit(srv, r)
        ready.release()
    th.join()
    _serve_run.last_wait = wait
    return lat, time.perf_counter() - t0


def _plain_run(R, torch, reqs, n_set):
    """The same requests as sequential plain calls (no resident states)."""
    buf = torch.empty(1 << 26, dtype=torch.int32, device="cuda")
    lat = []
    t0 = time.perf_counter()
    for r in reqs:
        ts = time.perf_counter()
        if r.type == R.RNG_REQ_DRAW:
            h = R.rng_create(r.kind, n_set)
            R.rng_seed(h, r.seed)
            if r.offset:
                R.rng_skipahead(h, r.offset)
            K = -(-r.count // n_set)
            if r.out == R.RNG_OUT_NORMAL:
                K += K % 2
            fn = {0: R.rng_generate_u32, 1: R.rng_generate_f32, 2: R.rng_generate_normal}[r.out]
            fn(h, buf.data_ptr(), K, R.RNG_STEP_MAJOR)
            torch.cuda.synchronize()
            R.rng_destroy(h)
        else:
            h = R.ising_create(r.L, r.beta, 0, r.kind, 0, r.seed, 2)
            R.ising_sweep(h, r.sweeps)
            R.ising_observables(h)
            R.ising_destroy(h)
        lat.append((time.perf_counter() - ts) * 1e3)
    return lat, time.perf_counter() - t0


def serve_section(R, torch, args):
    import numpy as np
    n_set = 4096
    reqs = serve_requests(R, args.serve_requests)
    numbers = sum(r.count for r in reqs if r.type == R.RNG_REQ_DRAW)
    srv = R.rng_server_create(512, n_set, 8, 16 << 30)
    try:
        _serve_run(R, srv, reqs[: min(40, len(reqs))], None)  # warm-up: sets, plans, ladders
        lat_cap, wall_cap = _serve_run(R, srv, reqs, None)  # closed loop: capacity
        cap = len(reqs) / wall_cap
        rates = {}
        is_sweep = np.array([r.type == R.RNG_REQ_SWEEP for r in reqs])
        for f in (0.5, 0.8, 1.0):
            lat, wall = _serve_run(R, srv, reqs, f * cap)
            lat_a, wait_a = np.array(lat), np.array(_serve_run.last_wait)
            rates[str(f)] = {"rate_req_s": round(f * cap, 1), "p50_ms": round(float(np.percentile(lat, 50)), 3),
                             "p99_ms": round(float(np.percentile(lat, 99)), 3),
                             "gnum_s": round(numbers / wall / 1e9, 2),
                             "p99_draw_ms": round(float(np.percentile(lat_a[~is_sweep], 99)), 3),
                             "p99_sweep_ms": round(float(np.percentile(lat_a[is_sweep], 99)), 3),
                             "p99_queue_wait_ms": round(float(np.percentile(wait_a, 99)), 3)}
        stats = R.rng_server_stats(srv)
    finally:
        R.rng_server_destroy(srv)
    lat_p, wall_p = _plain_run(R, torch, reqs, n_set)
    lat_pa = np.array(lat_p)
    return {"requests": len(reqs), "draw_numbers": numbers, "capacity_req_s": round(cap, 1),
            "capacity_gnum_s": round(numbers / wall_cap / 1e9, 2), "rates": rates,
            "plain_sequential": {"p50_ms": round(float(np.percentile(lat_p, 50)), 3),
                                 "p99_ms": round(float(np.percentile(lat_p, 99)), 3),
                                 "p99_draw_ms": round(float(np.percentile(lat_pa[~is_sweep], 99)), 3),
                                 "p99_sweep_ms": round(float(np.percentile(lat_pa[is_sweep], 99)), 3),
                                 "gnum_s": round(numbers / wall_p / 1e9, 2), "wall_s": round(wall_p, 2)},
            "speedup_vs_plain": round(wall_p / wall_cap, 2), "max_concurrent": stats["max_concurrent"],
            "workload": "80% draws (2^U(10,26) numbers, u32/f32/normal, 6 kinds, 64 seeds, offsets k 2^20), "
                        "20% sweeps (L in 64..1024, 10..1000 sweeps); 512 resident stream sets of 4096 "
                        "instances; 8 draw slots + 4 sweep slots; latency = submit to GPU completion"}


# ------------------------------------------------------------ CPU oracle arm
def oracle_sample(per_form: int, threads: int = 1):
    """Times the oracle on a bounded sample of the bulk workload: for every
    kind and form, per_form outputs (instances x draws like the GPU call).
    With threads > 1 the instances of each call are split into that many
    ranges run concurrently (the C oracle releases the interpreter lock)."""
    from concurrent.futures import ThreadPoolExecutor

    import numpy as np

    import oracle as O

    O.mwc_multipliers(8192)  # multiplier table outside the timed region
    pool = ThreadPoolExecutor(max_workers=threads) if threads > 1 else None

    def run(kind, form, n, K, i_lo, i_hi):
        r = O.generate(kind, SEED, n, K, i_lo=i_lo, i_hi=i_hi)
        if form == "f32":
            return O.to_f32(r)
        if form == "normal":
            return O.box_muller(r)
        if form == "u32_xor":
            return np.bitwise_xor.reduce(r, axis=1)
        return r

    total = 0
    t0 = time.perf_counter()
    for kind in range(N_KINDS):
        n = max(threads, 4 if kind in SHARED else 256)
        K = per_form // n
        for form in FORMS:
            if pool is None:
                run(kind, form, n, K, 0, n)
            else:
                cuts = [n * t // threads for t in range(threads + 1)]
                list(pool.map(lambda t: run(kind, form, n, K, cuts[t], cuts[t + 1]), range(threads)))
            total += n * K
    dt = time.perf_counter() - t0
    if pool is not None:
        pool.shutdown()
    return total, dt


def host_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(args):
    per_form = args.cpu_sample
    cores = host_threads()
    total1, dt1 = oracle_sample(per_form // 4)
    total, dt = 0, 0.0
    for _ in range(args.cpu_reps):  # about 10 s on all host threads
        t, d = oracle_sample(per_form, cores)
        total += t
        dt += d
    return {"value": round(total / dt / 1e9, 4), "unit": "Gnum/s", "cores": cores, "kind": "oracle",
            "single_thread": {"value": round(total1 / dt1 / 1e9, 4), "cores": 1,
                              "sample": f"{per_form // 4} outputs per kind and form, {dt1:.1f} s"},
            "sample": f"{args.cpu_reps} x {per_form} outputs per kind and form ({N_KINDS} kinds x 4 forms = "
                      f"{total} outputs), C oracle, instances split over {cores} threads, {dt:.1f} s"}


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return None
    per_form = args.cpu_sample
    cores = host_threads()
    oracle_sample(per_form // 8, cores)  # warm-up (builds and loads the oracle)
    times, total = [], 0
    for _ in range(args.warmup):
        oracle_sample(per_form // 4, cores)
    for _ in range(args.steps):
        tot, dt = oracle_sample(per_form // 4, cores)
        times.append(dt)
        total += tot
    v = total / sum(times) / 1e9
    return {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "Gnum/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * sum(times) / len(times), 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": bulk_config(world),
            "cpu_baseline": {"value": round(v, 4), "unit": "Gnum/s", "cores": cores, "kind": "oracle",
                             "sample": f"each step {per_form // 4} outputs per kind and form of the bulk workload "
                                       f"({total // len(times)} outputs), C oracle, instances split over {cores} "
                                       f"threads"},
            "e2e": {"value": round(v, 4), "unit": "Gnum/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ------------------------------------------------------- single-kernel cases
def run_case(args):
    """One kernel configuration on a small case, for a profiler: `gen` runs
    --reps calls of one generator kind and form; `ising` one persistent
    Ising launch (or multi-hit rounds with --hits); `all` one call of every
    kind and form of the bulk workload with its instance counts and
    --outputs / instances draws.  Prints "ok"."""
    import torch

    import paper_1204_6193_gb300 as R

    torch.cuda.set_device(0)
    kind = {v: k for k, v in R.KIND_NAMES.items()}[args.kind]
    if args.case == "all":
        out = torch.empty(args.outputs, dtype=torch.int32, device="cuda")
        for kd in sorted(R.KIND_NAMES):
            n = MT_GENS if kd in SHARED else N_INST
            K = args.outputs // n
            lay = R.RNG_INSTANCE_MAJOR if kd in SHARED else R.RNG_STEP_MAJOR
            h = R.rng_create(kd, n)
            R.rng_seed(h, SEED)
            R.rng_generate_u32(h, out.data_ptr(), K, lay)
            R.rng_generate_f32(h, out.data_ptr(), K, lay)
            R.rng_generate_normal(h, out.data_ptr(), K, lay)
            R.rng_generate_u32(h, out.data_ptr(), K, R.RNG_XOR_REDUCE)
            torch.cuda.synchronize()
            R.rng_destroy(h)
    elif args.case == "ising":
        layout = R.ISING_INT8 if args.spins == "int8" else R.ISING_MULTISPIN32
        h = R.ising_create(args.L, BETA_C, layout, kind, 0, SEED, 2)
        if args.launch:
            R.ising_set_launch(h, *(int(v) for v in args.launch.split(",")))
        if args.halo_depth is not None:
            R.ising_set_halo_depth(h, args.halo_depth)
        if args.hits:
            R.ising_sweep_multihit(h, args.sweeps, args.hits, args.strips)
        else:
            R.ising_sweep(h, args.sweeps)
        R.ising_observables(h)
        R.ising_destroy(h)
    else:
        layout = {"step": R.RNG_STEP_MAJOR, "instance": R.RNG_INSTANCE_MAJOR}[args.layout]
        h = R.rng_create(kind, args.n)
        R.rng_seed(h, SEED)
        out = torch.empty(args.n * (1 if args.form == "u32_xor" else args.K), dtype=torch.int32, device="cuda")
        for _ in range(args.reps):
            if args.form == "u32":
                R.rng_generate_u32(h, out.data_ptr(), args.K, layout)
            elif args.form == "f32":
                R.rng_generate_f32(h, out.data_ptr(), args.K, layout)
            elif args.form == "normal":
                R.rng_generate_normal(h, out.data_ptr(), args.K, layout)
            else:
                R.rng_generate_u32(h, out.data_ptr(), args.K, R.RNG_XOR_REDUCE)
        torch.cuda.synchronize()
        R.rng_destroy(h)
    print("ok")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-sample", type=int, default=1 << 24)
    ap.add_argument("--cpu-reps", type=int, default=16)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-ising", action="store_true")
    ap.add_argument("--ising-sweeps", type=int, default=100000)
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--batch-sweeps", type=int, default=10000)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=10000)
    # single-kernel cases for profiling (see run_case)
    ap.add_argument("--case", choices=["gen", "ising", "all"], default=None)
    ap.add_argument("--kind", default="lcg32")
    ap.add_argument("--form", default="u32", choices=["u32", "f32", "normal", "u32_xor"])
    ap.add_argument("--layout", default="step", choices=["step", "instance"])
    ap.add_argument("--n", type=int, default=1 << 20, help="instances (or warp-shared generators)")
    ap.add_argument("--K", type=int, default=64, help="draws per instance and call")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--L", type=int, default=1024, help="Ising lattice size")
    ap.add_argument("--spins", default="int8", choices=["int8", "multispin"])
    ap.add_argument("--sweeps", type=int, default=200, help="Ising sweeps (or multi-hit rounds)")
    ap.add_argument("--hits", type=int, default=0, help="k > 0: multi-hit rounds of k sweeps per strip phase")
    ap.add_argument("--strips", type=int, default=256)
    ap.add_argument("--launch", default="", help="threads,ctas_per_sm,min_sites_per_block of the Ising launch")
    ap.add_argument("--halo-depth", type=int, default=None, help="Ising exact checkerboard: 1 or 2 halo rows")
    ap.add_argument("--outputs", type=int, default=1 << 26, help="outputs per call with --case all")
    args = ap.parse_args()
    if args.case:
        run_case(args)
        return
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    line = run_reference(args) if args.impl == "reference" else run_gpu(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
