#!/usr/bin/env python3
"""Throughput benchmark: committed cell events per second of the exact parallel
simulator of the Poisson-asynchronous Glauber (continuous-time Ising) array.

Workload (one step): the 4096 x 4096 periodic Ising torus at beta = 0.30,
0.4407 and 0.60 (J = 1, h = 0, random +-1 initial spins from seed 7, Poisson
rate 1 per cell, 2^32 ticks per unit time), each initialised on the device and
run to T = 50 -- about 2.5e9 committed arrivals per step, all bit-exact against
the serial oracle (tests/).  The kernel and its tuning are picked by the
autotuner (on a GB300: the temporal-blocked round kernel).  The state
(3 x 201 MB) is larger than the 129 MB L2, so no flush is needed between steps.

Other workloads (--workload): batch (512 lattices, batched against plain calls),
serve (a replayed request stream) and frames (snapshot frames at K dt, B slots,
against the same run without frames).

Prints one JSON line (rank 0).  --impl reference times the CPU oracle on the
host cores on a bounded prefix of the same workload.
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

T32 = 1 << 32
BYTES_PER_EVENT = 26          # read + write of a cell's 13-byte state (int8 spin, int64 tick, uint32 count)
WORKLOAD = dict(name="ising4096x4096_T50", rows=4096, cols=4096, betas=[0.30, 0.4407, 0.60], J=1.0, h=0.0,
                seed=7, init=0, T=50)
CPU_SAMPLE_T = 0.5            # oracle sample: time prefix [0, 0.5) of the beta = 0.4407 lattice
ISSUE_PER_SM_CLK = 4          # one warp instruction per clock from each of an SM's four schedulers


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--kernel", default="round", choices=["blocked", "round", "epoch"])
    ap.add_argument("--lb", type=int, default=64)
    ap.add_argument("--rounds", type=int, default=8,
                    help="round kernel: synchronous rounds per launch (>1: temporal blocking); blocked: refresh")
    ap.add_argument("--polls", type=int, default=8)
    ap.add_argument("--per-lattice", action="store_true",
                    help="round kernel: run the lattices of a step one after another instead of as one batch")
    ap.add_argument("--no-autotune", action="store_true",
                    help="use --kernel/--lb/--rounds/--polls as given instead of the autotuned configuration")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the per-kernel side measurements")
    ap.add_argument("--workload", default="ising4096",
                    choices=["ising4096", "batch", "serve", "frames", "configs", "efficiency", "life", "rates",
                             "qnbhd", "sizes", "slabs"],
                    help="ising4096: the headline step; batch: the 512-lattice batch only; serve: the request stream")
    ap.add_argument("--serve-seconds", type=float, default=None,
                    help="length of the replayed request stream (default 60 s for --workload serve, 10 s in the "
                         "default run)")
    ap.add_argument("--single", action="store_true",
                    help="one lattice, one kernel configuration (the profiling case); prints one JSON line")
    ap.add_argument("--rows", type=int, default=4096)
    ap.add_argument("--cols", type=int, default=4096)
    ap.add_argument("--beta", type=float, default=0.4407)
    ap.add_argument("--T", type=float, default=5.0)
    return ap.parse_args()


def dist_env():
    from paper_cs_0502039_gb300.dist import rank_env
    return rank_env()


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _code_only(text):
    """Source text without comments, trailing blanks and empty lines: an edit that only
    changes comments leaves the compiled kernels, and so the committed profile, valid."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lines = (re.sub(r"//.*", "", ln).rstrip() for ln in text.splitlines())
    return "\n".join(ln for ln in lines if ln)


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("ac_kernels.cu", "ac_device.cuh"):
        with open(os.path.join(ROOT, "paper_cs_0502039_gb300", "csrc", f), encoding="utf-8") as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()


def committed_profile(kernel_name, key):
    """A per-step figure from the committed ncu summary, if it was taken on this kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    ent = rec.get(kernel_name)
    if not ent or ent.get("source_sha256") != kernel_source_hash():
        return None
    return ent.get(key)


def committed_traffic(kernel_name):
    """DRAM bytes per step (dram__bytes_read.sum + dram__bytes_write.sum)."""
    return committed_profile(kernel_name, "dram_bytes_per_step")


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


def cpu_baseline(sample_T=CPU_SAMPLE_T):
    import oracle
    w = WORKLOAD
    st = oracle.init(w["rows"], w["cols"], w["init"], w["seed"])
    thr = oracle.thresholds(0.4407, w["J"], w["h"])
    t0 = time.perf_counter()
    ev = oracle.run(st, thr, w["seed"], int(sample_T * T32))
    dt = time.perf_counter() - t0
    return {"value": ev / dt, "unit": "events/s", "cores": 1, "kind": "oracle",
            "sample": f"{w['rows']}x{w['cols']} beta=0.4407 seed {w['seed']}, arrivals in [0, {sample_T}) "
                      f"({ev} events, {dt:.1f} s, single-threaded C heap simulator)"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    w = WORKLOAD
    sample_T = 0.25
    times, evs = [], []
    for i in range(args.warmup + args.steps):
        st = oracle.init(w["rows"], w["cols"], w["init"], w["seed"])
        thr = oracle.thresholds(0.4407, w["J"], w["h"])
        t0 = time.perf_counter()
        ev = oracle.run(st, thr, w["seed"], int(sample_T * T32))
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
            evs.append(ev)
    value = sum(evs) / sum(times)
    sample = (f"{w['rows']}x{w['cols']} beta=0.4407 seed {w['seed']}, arrivals in [0, {sample_T}) per step "
              f"(~{evs[0]} events), single-threaded C heap oracle")
    out = {"metric": "cell_events_per_sec", "value": value, "unit": "events/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * sum(times) / len(times),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
           "data": "synthetic", "impl": "reference",
           "config": {"workload": w["name"], "rows": w["rows"], "cols": w["cols"], "betas": w["betas"],
                      "T": w["T"], "sample": sample},
           "cpu_baseline": {"value": value, "unit": "events/s", "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def kernel_id(ac, name):
    return {"blocked": ac.AC_KERNEL_BLOCKED, "round": ac.AC_KERNEL_ROUND, "epoch": ac.AC_KERNEL_EPOCH}[name]


def kernel_name(ac, kern):
    return {ac.AC_KERNEL_BLOCKED: "blocked", ac.AC_KERNEL_ROUND: "round", ac.AC_KERNEL_EPOCH: "epoch"}[kern]


def run_single(args):
    """One lattice (seed 7, random init, J = 1, h = 0) run to T with one kernel configuration:
    `warmup` untimed runs, then `steps` timed runs; reports the kernel's device time."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    import paper_cs_0502039_gb300 as ac
    kern = kernel_id(ac, args.kernel)
    with ac.Sim(args.rows, args.cols, args.beta, 1.0, 0.0, 7, kernel=kern, Lb=args.lb, rounds=args.rounds,
                polls=args.polls) as sim:
        for _ in range(args.warmup):
            sim.reset(7)
            sim.run_until(args.T)
        res = []
        for _ in range(args.steps):
            sim.reset(7)
            sim.run_until(args.T)
            res.append(sim.stats())
    ms = statistics.median(r["device_ms"] for r in res)
    ev = res[-1]["events"]
    print(json.dumps({"case": f"{args.rows}x{args.cols} beta={args.beta} T={args.T}", "kernel": args.kernel,
                      "Lb": args.lb, "rounds": args.rounds, "polls": args.polls, "events": ev,
                      "device_ms": ms, "events_per_s": ev / (ms / 1000.0),
                      "hbm_frac_effective": BYTES_PER_EVENT * ev / (ms / 1000.0) / 1e9 / measured_peaks()[0],
                      "launches": res[-1]["launches"], "visits": res[-1]["visits"], "polls_done": res[-1]["polls"],
                      "tile_rounds": res[-1]["rounds"], "scanned": res[-1]["scanned"],
                      "enabled_frac": res[-1]["enabled_frac_mean"], "checksum": res[-1]["checksum"]}),
          flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.single:
        return run_single(args)
    if args.workload == "configs":
        res = configs_measurement()
        print(json.dumps({"workload": args.workload, **res}), flush=True)
        return 0
    if args.workload == "sizes":
        import torch
        torch.cuda.set_device(0)
        import __graft_entry__
        __graft_entry__.build()
        import paper_cs_0502039_gb300 as ac
        print(json.dumps({"workload": args.workload, **sizes_measurement(ac)}), flush=True)
        return 0
    if args.workload == "qnbhd":
        import torch
        torch.cuda.set_device(0)
        import __graft_entry__
        __graft_entry__.build()
        import paper_cs_0502039_gb300 as ac
        print(json.dumps({"workload": args.workload, **qnbhd_measurement(ac)}), flush=True)
        return 0
    if args.workload == "rates":
        import torch
        torch.cuda.set_device(0)
        import __graft_entry__
        __graft_entry__.build()
        import paper_cs_0502039_gb300 as ac
        print(json.dumps({"workload": args.workload, **rates_measurement(ac)}), flush=True)
        return 0
    if args.workload == "life":
        import torch
        torch.cuda.set_device(0)
        import __graft_entry__
        __graft_entry__.build()
        import paper_cs_0502039_gb300 as ac
        print(json.dumps({"workload": args.workload, **life_measurement(ac)}), flush=True)
        return 0
    if args.workload == "efficiency":
        import torch
        torch.cuda.set_device(0)
        import __graft_entry__
        __graft_entry__.build()
        import paper_cs_0502039_gb300 as ac
        print(json.dumps({"workload": args.workload, **efficiency_measurement(ac)}), flush=True)
        return 0
    if args.workload == "slabs":
        import torch
        rank, world, local = dist_env()
        torch.cuda.set_device(local)
        if world > 1:
            import torch.distributed as tdist
            tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
        if rank == 0:
            import __graft_entry__
            __graft_entry__.build()
        if world > 1:
            tdist.barrier()
        import paper_cs_0502039_gb300 as ac
        res = slabs_measurement(ac, args.rounds)
        if rank == 0:
            print(json.dumps({"workload": args.workload, **res}), flush=True)
        if world > 1:
            tdist.destroy_process_group()
        return 0
    if args.workload in ("batch", "serve", "frames"):
        import torch
        torch.cuda.set_device(0)
        import __graft_entry__
        __graft_entry__.build()
        import paper_cs_0502039_gb300 as ac
        fixed = args.rounds if args.no_autotune else None
        if args.workload == "batch":
            res = batch_measurement(ac, fixed, args.lb)
        elif args.workload == "serve":
            res = serve_measurement(ac, args.serve_seconds or 60.0, fixed, args.lb)
        else:
            res = frames_measurement(ac, args.rounds, args.lb)
        print(json.dumps({"workload": args.workload, **res}), flush=True)
        return 0

    import numpy as np
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        dist = None

    if rank == 0:
        import __graft_entry__
        __graft_entry__.build()
    if dist:
        dist.barrier()
    import paper_cs_0502039_gb300 as ac

    w = WORKLOAD
    kern = kernel_id(ac, args.kernel)
    tuned = None
    if not args.no_autotune:
        # the step's own batch (three 4096^2 lattices), each candidate timed on the step's
        # horizon (shorter trials rank the epoch configurations by their start-up epochs)
        from paper_cs_0502039_gb300 import autotune
        tuned = autotune.tune_batch([(w["rows"], w["cols"], b) for b in w["betas"]], T=float(w["T"]))
        kern, args.lb, args.rounds, args.polls = tuned["kernel"], tuned["Lb"], tuned["rounds"], tuned["polls"]
        args.kernel = kernel_name(ac, kern)
    # weak scaling: every rank runs its own replica batch (seed offset by rank)
    from paper_cs_0502039_gb300.dist import replica_seed
    seed = replica_seed(w["seed"], rank)
    sims = [ac.Sim(w["rows"], w["cols"], b, w["J"], w["h"], seed, init=w["init"], kernel=kern, Lb=args.lb,
                   rounds=args.rounds, polls=args.polls) for b in w["betas"]]
    handles = [s.handle for s in sims]
    t_end = [w["T"] * T32] * len(sims)

    # the step's lattices run as one batch (one work list of all their tiles) or one after
    # another, as the autotuner found faster (--per-lattice: one after another)
    batched = kern == ac.AC_KERNEL_BLOCKED or not args.per_lattice
    if tuned is not None and not tuned.get("batched", True):
        batched = False

    def step():
        for s in sims:
            s.reset(seed, w["init"])
        if batched:
            ac.ac_batch_run_until(handles, t_end)
        else:
            for s in sims:
                s.run_until_ticks(t_end[0])

    def sync_all():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()

    # the trajectory is deterministic: every step commits the same arrivals, so the
    # per-step event count and the kernel's duration are read on passes outside the
    # timed region (stats() runs a reduction kernel)
    kern_ms_list, ev_step = [], None
    for _ in range(2):
        step()
        st = [s.stats() for s in sims]
        ev_step = sum(x["events"] for x in st)
        if batched:
            kern_ms_list.append(st[0]["device_ms"])          # one batched call (same on every handle)
        else:
            kern_ms_list.append(sum(x["device_ms"] for x in st))
    # init per lattice, then: blocked = publish + one kernel; batched round = count-range check +
    # the launches over all lattices' tiles; per lattice = count-range check + its launches
    if kern == ac.AC_KERNEL_BLOCKED:
        launches_per_step = len(sims) + 2
    elif batched:
        launches_per_step = len(sims) + 1 + st[0]["launches"]
    else:
        launches_per_step = sum(2 + x["launches"] for x in st)

    sync_all()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        start.record()
        for _ in range(args.steps):
            step()
        stop.record()
        torch.cuda.synchronize()
    ev_total = ev_step * args.steps
    launches = launches_per_step * args.steps
    kern_ms = statistics.median(kern_ms_list) * args.steps
    elapsed_ms = start.elapsed_time(stop)
    if dist:
        t = torch.tensor([elapsed_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())
        e = torch.tensor([float(ev_total)], device="cuda", dtype=torch.float64)
        dist.all_reduce(e)
        ev_all = float(e.item())
    else:
        ev_all = float(ev_total)
    value = ev_all / (elapsed_ms / 1000.0)
    ev_per_step_rank = ev_total / args.steps

    # roofline of the dominant kernel: algorithmic bytes per launch / its CUDA-event duration
    peak, peak_src = measured_peaks()
    kern_launch_ms = kern_ms / args.steps
    achieved = BYTES_PER_EVENT * ev_per_step_rank / (kern_launch_ms / 1000.0) / 1e9
    region = 96 if args.rounds <= 12 and args.lb != 128 else 128
    if kern == ac.AC_KERNEL_BLOCKED:
        kname = f"blocked_kernel<{args.lb}>"
    elif kern == ac.AC_KERNEL_EPOCH:
        kname = f"tb_kernel<{region},EP> rounds={args.rounds}" + (" batched" if batched else "")
    elif args.rounds > 1:
        kname = f"tb_kernel<{region}> rounds={args.rounds}" + (" batched" if batched else "")
    else:
        kname = f"round_kernel<{args.lb}>"
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": committed_traffic(kname), "peak_source": peak_src,
                "kernel": kname, "bytes_per_event": BYTES_PER_EVENT,
                "events_per_launch": ev_per_step_rank, "launch_ms": kern_launch_ms}
    # the kernel is bound by integer issue, not by DRAM: executed warp instructions per step (ncu
    # sm__inst_executed.sum on this source) over the live kernel time, against every scheduler
    # issuing one warp instruction per clock at the maximum SM clock
    inst = committed_profile(kname, "warp_inst_per_step")
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    clk_max = clk.summary()["sm_max_mhz"] or 2070.0
    issue_peak = ISSUE_PER_SM_CLK * n_sm * clk_max * 1e6 / 1e9
    issue = {"bound": "alu", "unit": "Gwarp-inst/s", "peak": issue_peak, "achieved": None, "frac": None,
             "peak_source": f"{ISSUE_PER_SM_CLK} x {n_sm} SMs x {clk_max:.0f} MHz",
             "warp_inst_per_event": None if inst is None else inst / ev_per_step_rank}
    if inst is not None:
        issue["achieved"] = inst / (kern_launch_ms / 1000.0) / 1e9
        issue["frac"] = issue["achieved"] / issue_peak

    # end-to-end through the public API with host buffers (pinned), copies inside the timed region
    e2e = None
    if not args.no_e2e:
        N = w["rows"] * w["cols"]
        init_state = []
        for s in sims:
            s.reset(seed, w["init"])
            host = (torch.empty(N, dtype=torch.int8).pin_memory(), torch.empty(N, dtype=torch.int64).pin_memory(),
                    torch.empty(N, dtype=torch.int32).pin_memory())
            ac.ac_read_state(s.handle, host[0].numpy(), host[1].numpy(), host[2].numpy().view(np.uint32))
            init_state.append(host)
        outs = [(torch.empty(N, dtype=torch.int8).pin_memory(), torch.empty(N, dtype=torch.int64).pin_memory(),
                 torch.empty(N, dtype=torch.int32).pin_memory()) for _ in sims]
        # lattices run one after another on a compute stream; their pinned-host loads and reads
        # go on a copy stream, so that lattice i+1 is loaded and lattice i-1 read back while
        # lattice i runs (the handle's own transfers never overlap its own runs)
        compute, copy = torch.cuda.Stream(), torch.cuda.Stream()
        for s in sims:
            ac.ac_set_stream(s.handle, compute.cuda_stream)
        views = [(hs.numpy(), ht.numpy(), hn.numpy().view(np.uint32)) for hs, ht, hn in init_state]
        oviews = [(a.numpy(), b.numpy(), c.numpy().view(np.uint32)) for a, b, c in outs]

        def e2e_run(steps):
            """`steps` steps as one stream of (step, lattice) jobs: while job j runs, job j+1 is loaded
            and job j-1 read back; every job's load and read is inside the timed region."""
            jobs = [i for _ in range(steps) for i in range(len(sims))]
            ac.ac_load_state_async(sims[jobs[0]].handle, *views[jobs[0]], 0, copy.cuda_stream)
            for j, i in enumerate(jobs):
                if j + 1 < len(jobs):
                    # the next job's handle (another lattice, or this step's first one again) was
                    # read back in an earlier job; its load waits on the device for that read
                    ac.ac_load_state_async(sims[jobs[j + 1]].handle, *views[jobs[j + 1]], 0, copy.cuda_stream)
                sims[i].run_until_ticks(t_end[i])
                ac.ac_read_state_async(sims[i].handle, *oviews[i], copy.cuda_stream)
            copy.synchronize()

        e2e_run(1)                        # untimed: events and staging of the asynchronous path
        sync_all()
        e_steps = max(1, min(args.steps, 3))
        t0 = time.perf_counter()
        e2e_run(e_steps)
        torch.cuda.synchronize()
        e_dt = time.perf_counter() - t0
        # the trajectory is deterministic: every step commits the device-timed step's arrivals;
        # checked on the results the last step read back (outside the timed region)
        got = sum(int(on.numpy().view(np.uint32).astype(np.int64).sum()) for _, _, on in outs)
        if got != ev_per_step_rank:
            raise RuntimeError(f"end-to-end run committed {got} arrivals, the device-timed step {ev_per_step_rank}")
        e_ev = ev_per_step_rank * e_steps
        if dist:
            t = torch.tensor([e_dt], device="cuda", dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e_dt = float(t.item())
            e = torch.tensor([float(e_ev)], device="cuda", dtype=torch.float64)
            dist.all_reduce(e)
            e_ev = e.item()
        # per lattice and direction: spins int8 + ticks int64 + counts uint32 = 13 bytes per cell
        e2e = {"value": e_ev / e_dt, "unit": "events/s", "h2d_bytes_per_step": 13 * N * len(sims),
               "d2h_bytes_per_step": 13 * N * len(sims), "steps": e_steps,
               "path": "per lattice and step: ac_load_state_async (pinned host, copy stream), ac_run_until_ticks "
                       "(compute stream), ac_read_state_async (pinned host, copy stream); the steps' lattices form one "
                       "stream of jobs, the next job loading and the previous one reading back while a job runs",
               "over_device": (e_ev / e_dt) / value}
        for s in sims:
            ac.ac_set_stream(s.handle, None)

    extra, batch, served = {}, None, None
    if rank == 0 and not args.no_extra:
        extra = side_measurements(ac, w, seed)
        batch = batch_measurement(ac)
        served = serve_measurement(ac, seconds=args.serve_seconds or 10.0)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline()

    stats0 = sims[0].stats()
    for s in sims:
        s.close()
    if rank == 0:
        out = {"metric": "cell_events_per_sec", "value": value, "unit": "events/s", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
               "data": "synthetic",
               "config": {"workload": w["name"], "rows": w["rows"], "cols": w["cols"], "betas": w["betas"],
                          "J": w["J"], "h": w["h"], "seed": w["seed"], "T": w["T"], "init": "random",
                          "kernel": kname, "Lb": args.lb, "polls": args.polls, "rounds": args.rounds,
                          "autotuned": None if tuned is None else {k: tuned[k] for k in ("kernel", "Lb", "rounds",
                                                                                       "polls", "batched",
                                                                                       "events_per_s", "measured")
                                                                  if k in tuned},
                          "batched": batched,
                          "events_per_step": ev_all / args.steps,
                          "l2": "state 3 x 201 MB > 129 MB L2 (no flush)",
                          "parallelism": f"replicas x{world}"},
               "roofline": roofline, "roofline_issue": issue, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
               "clocks": clk.summary(),
               "kernel_stats": {k: stats0[k] for k in ("visits", "polls", "rounds", "scanned", "enabled",
                                                       "grid", "ctas_per_sm")},
               "kernels": extra, "batch": batch, "serve": served}
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def batch_measurement(ac, rounds=None, lb=64):
    """512 independent lattices (L log-uniform in [32, 1024], beta ~ U[0.3, 0.6], seeds 0..511) run
    to T = 100: one batched call (one work list of all tiles) against 512 plain per-lattice run
    calls on the same GPU, both with the configuration the autotuner picks for this batch (or
    `rounds` rounds per launch of the round kernel).  Every lattice's state fingerprint must be
    the same in both modes."""
    from paper_cs_0502039_gb300 import autotune, workloads
    ws = workloads.batch_workload()
    if rounds is None:
        cfg = autotune.tune_batch([(w["rows"], w["cols"], w["beta"]) for w in ws], T=5.0, batched_only=True)
    else:
        cfg = dict(kernel=ac.AC_KERNEL_ROUND, Lb=lb, rounds=rounds, polls=8)
    handles = ac.ac_batch_create([(w["rows"], w["cols"], w["init"]) for w in ws], [w["beta"] for w in ws],
                                 [w["J"] for w in ws], [w["h"] for w in ws], [w["seed"] for w in ws])
    sims = [ac.Sim(w["rows"], w["cols"], w["beta"], w["J"], w["h"], w["seed"], handle=h) for w, h in zip(ws, handles)]
    for s in sims:
        s.configure(cfg["kernel"], cfg["Lb"], cfg["rounds"], max(cfg["polls"], 0))
    t_end = [int(w["T"] * T32) for w in ws]
    import torch

    def reset_all():
        for w, s in zip(ws, sims):
            s.reset(w["seed"], w["init"])

    out = {"lattices": len(ws), "cells": sum(w["rows"] * w["cols"] for w in ws), "T": ws[0]["T"],
           "config": {"kernel": kernel_name(ac, cfg["kernel"]), "Lb": cfg["Lb"], "rounds": cfg["rounds"],
                      "tuned": rounds is None}}
    prints = {}
    for mode in ("batched", "plain"):
        times = []
        for rep in range(3):          # rep 0 warms up (and, for batched, captures the graph)
            reset_all()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if mode == "batched":
                ac.ac_batch_run_until([s.handle for s in sims], t_end)
            else:
                for s, te in zip(sims, t_end):
                    s.run_until_ticks(te)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        st = [s.stats() for s in sims]
        prints[mode] = [(x["checksum"], x["total_counts"], x["sum_s"], x["sum_bonds"]) for x in st]
        ev = sum(x["events"] for x in st)
        out[mode] = {"events": ev, "seconds": min(times[1:]), "events_per_s": ev / min(times[1:])}
    same = sum(a == b for a, b in zip(prints["batched"], prints["plain"]))
    out["per_lattice_equal"] = f"{same}/{len(ws)}"
    if same != len(ws):
        raise RuntimeError(f"batched and plain runs differ on {len(ws) - same} lattices")
    out["batched_over_plain"] = out["batched"]["events_per_s"] / out["plain"]["events_per_s"]
    for s in sims:
        s.close()
    return out


def serve_measurement(ac, seconds=10.0, rounds=None, lb=64):
    """Continuous batching: a Poisson request stream (200 requests/s, L log-uniform in [64, 2048],
    beta ~ U[0.25, 0.7], T ~ U[10, 200], seed = request id) replayed in real time; latency is
    request arrival -> result ready.  Then the same request set with every request visible at
    once (the server's capacity), and, as the baseline, the same request set run one request
    after another, each with its own plain run call, on the same GPU.  The configuration is
    the autotuner's for a batch of the stream's first 64 lattices (or `rounds` rounds per
    launch of the round kernel)."""
    from paper_cs_0502039_gb300 import autotune
    from paper_cs_0502039_gb300 import serve as srv_mod
    from paper_cs_0502039_gb300 import workloads
    reqs = workloads.serve_requests(rate=200.0, duration=seconds)
    if rounds is None:
        cfg = autotune.tune_batch([(r["rows"], r["cols"], r["beta"]) for r in reqs[:64]], T=5.0, batched_only=True)
    else:
        cfg = dict(kernel=ac.AC_KERNEL_ROUND, Lb=lb, rounds=rounds, polls=8)
    kw = dict(budget_bytes=64 << 30, slice_T=10.0, kernel=cfg["kernel"], rounds=cfg["rounds"], Lb=cfg["Lb"])
    results, wall, server = srv_mod.serve(reqs, realtime=True, **kw)
    lat = sorted(r.latency for r in results)
    ev = sum(r.events for r in results)
    span = max(r.finished for r in results) - min(r.arrival for r in results)
    out = {"requests": len(reqs), "seconds": seconds, "rate_per_s": 200.0, "completed": len(results), "wall_s": wall,
           "config": {"kernel": kernel_name(ac, cfg["kernel"]), "Lb": cfg["Lb"], "rounds": cfg["rounds"]},
           "events": ev, "events_per_s": ev / span, "p50_latency_s": lat[len(lat) // 2],
           "p99_latency_s": lat[min(len(lat) - 1, int(0.99 * len(lat)))], "steps": server.steps,
           "offered_events_per_s": sum(r["rows"] * r["cols"] * r["T"] for r in reqs) / seconds}
    # capacity: the same requests, all visible at t = 0
    sat, sat_wall, sat_server = srv_mod.serve(reqs, realtime=False, **kw)
    sat_ev = sum(r.events for r in sat)
    if [(r.id, r.checksum) for r in sat] != [(r.id, r.checksum) for r in results]:
        raise RuntimeError("the saturated serve run differs from the real-time one")
    out["saturated"] = {"events": sat_ev, "wall_s": sat_wall, "events_per_s": sat_ev / sat_wall,
                        "steps": sat_server.steps}
    # serial per-request baseline over the same request set, timed end to end
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sev = 0
    for r in reqs:
        with ac.Sim(r["rows"], r["cols"], r["beta"], r["J"], r["h"], r["seed"], init=r["init"],
                    kernel=cfg["kernel"], Lb=cfg["Lb"], rounds=cfg["rounds"]) as s:
            s.run_until(r["T"])
            sev += s.stats()["events"]
    dt = time.perf_counter() - t0
    out["serial"] = {"requests": len(reqs), "events": sev, "events_per_s": sev / dt, "seconds": dt}
    out["capacity_over_serial"] = out["saturated"]["events_per_s"] / out["serial"]["events_per_s"]
    return out


def slabs_measurement(ac, rounds=8):
    """One 4096^2 lattice (beta 0.4407, seed 7, T = 50) split into row slabs.  In one process
    (one GPU) the slabs are handles stepped one after another with halo rows copied between
    them; under torchrun each rank holds one slab and the halo rows go over torch.distributed
    (NCCL).  The fingerprint of the assembled state must equal the unsplit run's."""
    import torch
    from paper_cs_0502039_gb300 import slabs
    rank, world, _ = dist_env()
    w = WORKLOAD
    t_end = w["T"] * T32
    with ac.Sim(w["rows"], w["cols"], 0.4407, w["J"], w["h"], w["seed"], init=w["init"],
                kernel=ac.AC_KERNEL_ROUND, Lb=64, rounds=rounds) as ref:
        ref.run_until(w["T"])
        want = ref.stats()["checksum"]
    out = {"lattice": f"{w['rows']}x{w['cols']}", "beta": 0.4407, "T": w["T"], "rounds": rounds, "cases": []}

    def gather(sims, plan):
        for sim, sl in zip(sims[1:], plan[1:]):
            buf = torch.empty(sl.nrows * w["cols"] * 12, dtype=torch.uint8, device="cuda")
            ac.ac_slab_export(sim.handle, sl.row0, sl.nrows, buf.data_ptr())
            ac.ac_slab_import(sims[0].handle, sl.row0, sl.nrows, buf.data_ptr())
        return sims[0].stats()["checksum"]

    if world == 1:
        for nslabs in (2, 4):
            plan = slabs.plan(w["rows"], nslabs, rounds)
            sims = [ac.Sim(w["rows"], w["cols"], 0.4407, w["J"], w["h"], w["seed"], init=w["init"],
                           kernel=ac.AC_KERNEL_ROUND, Lb=64, rounds=rounds) for _ in plan]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            steps = slabs.run_on_one_gpu(ac, sims, plan, rounds, t_end)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            ev = sum(x.stats()["events"] for x in sims)
            ok = gather(sims, plan) == want
            for x in sims:
                x.close()
            out["cases"].append({"slabs": nslabs, "ranks": 1, "steps": steps, "events": ev, "seconds": dt,
                                 "events_per_s": ev / dt, "checksum_equal": ok})
            if not ok:
                raise RuntimeError(f"{nslabs} slabs: the assembled state differs from the unsplit run")
    else:
        import torch.distributed as tdist
        sim = ac.Sim(w["rows"], w["cols"], 0.4407, w["J"], w["h"], w["seed"], init=w["init"],
                     kernel=ac.AC_KERNEL_ROUND, Lb=64, rounds=rounds)
        tdist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        steps = slabs.run_distributed(ac, sim, rank, world, rounds, t_end)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        ev = torch.tensor([float(sim.stats()["events"])], device="cuda", dtype=torch.float64)
        tm = torch.tensor([dt], device="cuda", dtype=torch.float64)
        tdist.all_reduce(ev)
        tdist.all_reduce(tm, op=tdist.ReduceOp.MAX)
        sim.close()
        out["cases"].append({"slabs": world, "ranks": world, "steps": steps, "events": ev.item(),
                             "seconds": tm.item(), "events_per_s": ev.item() / tm.item()})
    return out


def frames_measurement(ac, rounds=6, lb=64):
    """Snapshot frames (Fig. 3.7) on the 4096^2 beta = 0.4407 lattice to T = 50: arrivals per second
    of the run with frames every dt time units in B slots (frames written by the kernels and dropped,
    or copied to the host), against the same run without frames.  The trajectory is the same in
    every case (tests/test_gpu_frames.py); what changes is the lag bound of B dt time units."""
    import torch
    w = WORKLOAD
    out = {"lattice": f"{w['rows']}x{w['cols']}", "beta": 0.4407, "T": w["T"], "rounds": rounds, "cases": []}
    with ac.Sim(w["rows"], w["cols"], 0.4407, w["J"], w["h"], w["seed"], init=w["init"], kernel=ac.AC_KERNEL_ROUND,
                Lb=lb, rounds=rounds) as sim:
        def timed(dt_units, B, mode):
            best, ev = None, 0
            for _ in range(2):           # the first pass warms up
                sim.reset(w["seed"], w["init"])
                if B:
                    sim.configure_frames(int(dt_units * T32), 0, B)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                if not B:
                    sim.run_until(w["T"])
                elif mode == "host":
                    got = [0]

                    def fn(K, ptr, n):
                        got[0] += 1
                    ac.ac_run_until_frames(sim.handle, w["T"] * T32, fn, on_host=True)
                else:
                    ac.ac_run_until_frames(sim.handle, w["T"] * T32, None)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                ev = sim.stats()["events"]
                best = dt if best is None else min(best, dt)
            return ev, best

        ev0, t0 = timed(0, 0, None)
        out["no_frames"] = {"events": ev0, "seconds": t0, "events_per_s": ev0 / t0}
        # the lag bound B dt (in mean interarrival times), as in the paper's bounded-lag experiment
        for lag, B, mode in [(0.3, 1, "drop"), (1.0, 1, "drop"), (2.0, 1, "drop"), (4.0, 1, "drop"),
                             (8.0, 1, "drop"), (16.0, 1, "drop"), (1.0, 4, "drop"), (4.0, 4, "drop"),
                             (16.0, 4, "drop"), (16.0, 16, "drop"), (4.0, 4, "host")]:
            dt_units = lag / B
            ev, t = timed(dt_units, B, mode)
            assert ev == ev0
            out["cases"].append({"lag": lag, "dt": dt_units, "B": B, "frames": int(w["T"] / dt_units), "mode": mode,
                                 "seconds": t, "events_per_s": ev / t, "relative": t0 / t})
    return out


def sizes_measurement(ac):
    """Single-lattice throughput against the lattice side L (beta 0.4407, random start from seed 7):
    the temporal-blocked round kernel at 6 rounds per launch, the blocked kernel with tiles of 64 and
    128, and the autotuner's choice for the size class.  T is chosen so that a run is a few tens of
    milliseconds or more."""
    import torch
    from paper_cs_0502039_gb300 import autotune
    R, B = ac.AC_KERNEL_ROUND, ac.AC_KERNEL_BLOCKED
    out = {"beta": 0.4407, "cases": []}
    for L, T in ((256, 200), (512, 100), (1024, 50), (2048, 50), (4096, 50), (8192, 10), (16384, 5)):
        tuned = autotune.tune(L, L)
        row = {"L": L, "T": T, "autotuned_config": {k: tuned[k] for k in ("kernel", "Lb", "rounds", "polls")}}
        for name, kern, lb, rounds, polls in (("round_r6", R, 64, 6, 0), ("blocked_lb64", B, 64, 1, 8),
                                              ("blocked_lb128", B, 128, 1, 8),
                                              ("autotuned", tuned["kernel"], tuned["Lb"], tuned["rounds"],
                                               tuned["polls"])):
            with ac.Sim(L, L, 0.4407, 1.0, 0.0, 7, kernel=kern, Lb=lb, rounds=rounds, polls=polls) as sim:
                sim.run_until(min(T, 2))
                sim.reset(7)
                torch.cuda.synchronize()
                sim.run_until(T)
                st = sim.stats()
            row[name] = {"events_per_s": st["events"] / (st["device_ms"] / 1000.0), "device_ms": st["device_ms"]}
        out["cases"].append(row)
    return out


def qnbhd_measurement(ac):
    """The Ising array on the q-th degree neighbourhood (Sec. 3) on a 4096^2 torus, random start
    (seed 7), beta 0.15, run to T = 50 with the temporal-blocked kernel, for q = 1, 2, 3."""
    import torch
    w = WORKLOAD
    out = {"lattice": f"{w['rows']}x{w['cols']}", "beta": 0.15, "T": w["T"], "cases": []}
    for q, rounds in ((1, 6), (2, 3), (3, 2), (2, 6), (3, 4)):
        if q == 1:
            sim = ac.Sim(w["rows"], w["cols"], 0.15, 1.0, 0.0, w["seed"], kernel=ac.AC_KERNEL_ROUND, Lb=64,
                         rounds=rounds)
        else:
            sim = ac.ising_q(w["rows"], w["cols"], 0.15, q, seed=w["seed"], rounds=rounds)
        with sim:
            sim.run_until(w["T"])
            sim.reset(w["seed"], 0)
            torch.cuda.synchronize()
            sim.run_until(w["T"])
            st = sim.stats()
        out["cases"].append({"q": q, "neighbours": 2 * q * (q + 1), "rounds_per_launch": rounds, "halo": q * rounds,
                             "events": st["events"], "device_ms": st["device_ms"],
                             "events_per_s": st["events"] / (st["device_ms"] / 1000.0)})
    return out


def rates_measurement(ac, rounds=6):
    """Per-cell rates (law (A) of Sec. 2) on the 4096^2 beta = 0.4407 lattice to T = 50: rate
    multipliers drawn log-uniformly so that rates span 1/8 .. 8 (seed 5), against rate 1."""
    import numpy as np
    import torch
    w = WORKLOAD
    N = w["rows"] * w["cols"]
    rng = np.random.default_rng(5)
    m = np.exp(rng.uniform(np.log(ac.AC_RATE_ONE / 8), np.log(ac.AC_RATE_ONE * 8), N)).astype(np.uint32)
    out = {"lattice": f"{w['rows']}x{w['cols']}", "beta": 0.4407, "T": w["T"], "rounds": rounds, "cases": []}
    for name, rates in (("rate 1", None), ("rates 1/8 .. 8", m)):
        with ac.Sim(w["rows"], w["cols"], 0.4407, w["J"], w["h"], w["seed"], init=w["init"],
                    kernel=ac.AC_KERNEL_ROUND, Lb=64, rounds=rounds) as sim:
            sim.set_rates(rates)
            sim.run_until(w["T"])
            sim.reset(w["seed"], w["init"])
            torch.cuda.synchronize()
            sim.run_until(w["T"])
            st = sim.stats()
        out["cases"].append({"case": name, "events": st["events"], "device_ms": st["device_ms"],
                             "events_per_s": st["events"] / (st["device_ms"] / 1000.0)})
    return out


def life_measurement(ac):
    """Asynchronous Conway Life (B3/S23, Moore neighbourhood) on a 4096^2 torus, half the cells
    alive at the start (seed 7), run to T = 50 with the temporal-blocked kernel: committed arrivals
    per second for several rounds per launch, beside the Ising array on the same kernel."""
    import torch
    w = WORKLOAD
    out = {"lattice": f"{w['rows']}x{w['cols']}", "rule": "B3/S23", "density": 0.5, "T": w["T"], "cases": []}
    for rounds in (4, 6, 8):
        with ac.life(w["rows"], w["cols"], w["seed"], 0.5, rounds=rounds) as sim:
            sim.run_until(w["T"])
            sim.reset(w["seed"], 0)
            torch.cuda.synchronize()
            sim.run_until(w["T"])
            st = sim.stats()
            s, _, _ = sim.read_state()
        out["cases"].append({"rounds": rounds, "events": st["events"], "device_ms": st["device_ms"],
                             "events_per_s": st["events"] / (st["device_ms"] / 1000.0),
                             "alive_fraction_at_T": float((s > 0).mean())})
    return out


def efficiency_measurement(ac, rounds=2000):
    """Sec. 4's time-only round model at large sizes: the fraction of cells that advance per
    round (mean over the second half of `rounds` rounds), for a 2^24-cell circle, a 4096^2 torus
    and a 256^3 periodic array, each with exponential, uniform and r^(1/8) increments, beside the
    limits the paper reports; and the rate of cell advances on the GPU."""
    import numpy as np
    paper = {(1, 0): 0.247, (1, 1): 0.271, (1, 2): 0.3388, (2, 0): 0.121, (2, 1): 0.132}
    out = {"rounds": rounds, "cases": []}
    for dims, n in [(1, 1 << 24), (2, 4096), (3, 256)]:
        for law, name in [(ac.AC_LAW_EXP, "exponential"), (ac.AC_LAW_UNIFORM, "uniform"), (ac.AC_LAW_ROOT8, "r^(1/8)")]:
            en, _, _, ms = ac.ac_time_model(dims, n, law, 11, 2**61 - 1, rounds)
            N = n ** dims
            frac = en.astype(np.float64) / N
            out["cases"].append({"dims": dims, "n": n, "law": name, "efficiency": float(frac[rounds // 2:].mean()),
                                 "efficiency_first_round": float(frac[0]), "paper": paper.get((dims, law)),
                                 "advances": int(en.sum()), "device_ms": ms,
                                 "advances_per_s": float(en.sum()) / (ms / 1000.0)})
    # the q-th degree neighbourhood of Sec. 3: a cell waits for every cell within distance q
    out["q_neighbourhood"] = []
    for q in (1, 2, 3, 4):
        en, _, _, ms = ac.ac_time_model(2, 4096, ac.AC_LAW_EXP, 11, 2**61 - 1, rounds, q=q)
        frac = en.astype(np.float64) / 4096 ** 2
        out["q_neighbourhood"].append({"dims": 2, "n": 4096, "q": q, "neighbours": 2 * q * (q + 1),
                                       "efficiency": float(frac[rounds // 2:].mean()),
                                       "efficiency_first_round": float(frac[0]), "device_ms": ms})
    return out


def _oracle_batch_prefix(items):
    """CPU-baseline worker: oracle runs of a list of (rows, cols, init, seed, beta, t_end)."""
    import oracle
    ev = 0
    for rows, cols, init, seed, beta, t_end in items:
        st = oracle.init(rows, cols, init, seed)
        ev += oracle.run(st, oracle.thresholds(beta), seed, t_end)
    return ev


def configs_measurement():
    """Numbers for the smaller and larger configurations beside the main workload.
    C1: 64x64, random init from seed 1, beta 0.44, T = 10 (every kernel; the oracle's full run).
    C3: 16384x16384, all up, seed 3, beta 1.0, h 0.05, T = 20 (the autotuned kernel and each tile side
        of the blocked kernel; the oracle on the prefix [0, 0.05)).
    C4: the oracle over the 512-lattice batch on all host cores, prefix [0, 1) of every lattice
        (the GPU numbers of C4 and C5 come from --workload batch / serve).
    The oracle's process pool is started before the first GPU call."""
    import multiprocessing as mp
    import __graft_entry__
    __graft_entry__.build()          # compiles and loads the library; no GPU call yet
    import oracle
    from paper_cs_0502039_gb300 import workloads
    ws = workloads.batch_workload()
    cores = os.cpu_count() or 1
    items = [(w["rows"], w["cols"], w["init"], w["seed"], w["beta"], T32) for w in ws]
    chunks = [items[i::cores] for i in range(cores)]
    with mp.get_context("spawn").Pool(cores) as pool:
        t0 = time.perf_counter()
        ev = sum(pool.map(_oracle_batch_prefix, chunks))
        dt = time.perf_counter() - t0
    out = {"c4_oracle": {"events": ev, "seconds": dt, "events_per_s": ev / dt, "cores": cores,
                         "sample": "all 512 lattices, arrivals in [0, 1), one process per core"}}

    st = oracle.init(64, 64, 0, 1)
    t0 = time.perf_counter()
    ev = oracle.run(st, oracle.thresholds(0.44), 1, 10 * T32)
    dt = time.perf_counter() - t0
    out["c1_oracle"] = {"events": ev, "seconds": dt, "events_per_s": ev / dt, "cores": 1}
    st = oracle.init(16384, 16384, 1, 3)
    t0 = time.perf_counter()
    ev = oracle.run(st, oracle.thresholds(1.0, 1.0, 0.05), 3, int(0.05 * T32))
    dt = time.perf_counter() - t0
    out["c3_oracle"] = {"events": ev, "seconds": dt, "events_per_s": ev / dt, "cores": 1,
                        "sample": "arrivals in [0, 0.05)"}
    del st

    import torch
    torch.cuda.set_device(0)
    import paper_cs_0502039_gb300 as ac
    from paper_cs_0502039_gb300 import autotune
    R, B = ac.AC_KERNEL_ROUND, ac.AC_KERNEL_BLOCKED

    def measure(rows, cols, init, seed, beta, h, T, kern, lb, rounds, polls, warm_T, early=0):
        with ac.Sim(rows, cols, beta, 1.0, h, seed, init=init, kernel=kern, Lb=lb, rounds=rounds, polls=polls) as s:
            if early:
                s.set_option(ac.AC_OPT_EARLY_REJECT, 1)
            s.run_until(warm_T)
            s.reset(seed, init)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s.run_until(T)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            st = s.stats()
        return {"kernel": kernel_name(ac, kern), "Lb": lb, "rounds": rounds, "polls": polls,
                "early_reject": bool(early), "early_commits": st["early_commits"], "launches": st["launches"],
                "events": st["events"], "device_ms": st["device_ms"], "wall_ms": 1000 * wall,
                "events_per_s": st["events"] / (st["device_ms"] / 1000.0),
                "hbm_frac_effective": BYTES_PER_EVENT * st["events"] / (st["device_ms"] / 1000.0) / 1e9
                / measured_peaks()[0]}

    out["c1"] = [measure(64, 64, 0, 1, 0.44, 0.0, 10, k, lb, r, p, 10)
                 for k, lb, r, p in [(R, 32, 1, 0), (R, 64, 4, 0), (B, 32, 1, 8), (B, 64, 1, 8)]]
    tuned = autotune.tune(16384, 16384)
    cfgs = [(tuned["kernel"], tuned["Lb"], tuned["rounds"], tuned["polls"]), (R, 64, 6, 0),
            (B, 32, 1, 8), (B, 64, 1, 8), (B, 128, 1, 8)]
    out["c3"] = [measure(16384, 16384, 1, 3, 1.0, 0.05, 20, k, lb, r, p, 1) for k, lb, r, p in cfgs]
    # BKL on / off: the one-round kernel (one synchronous round of Fig. 3.2 per launch) with and
    # without early commits of certain rejections
    out["c3_bkl"] = [measure(16384, 16384, 1, 3, 1.0, 0.05, 20, R, 64, 1, 0, 1, early) for early in (0, 1)]
    out["c2_bkl"] = [measure(4096, 4096, 0, 7, 0.4407, 0.0, 50, R, 64, 1, 0, 1, early) for early in (0, 1)]
    out["c3_autotuned"] = {k: tuned[k] for k in ("kernel", "Lb", "rounds", "polls")}
    return out


def side_measurements(ac, w, seed):
    """Single-lattice numbers for each kernel (beta = 0.4407 lattice, one run each)."""
    res = {}
    configs = [("round_r1_lb64", ac.AC_KERNEL_ROUND, 64, 1, 0), ("round_r8_lb64", ac.AC_KERNEL_ROUND, 64, 8, 0),
               ("blocked_epoch_r8", ac.AC_KERNEL_EPOCH, 64, 8, 0), ("blocked_epoch_r10", ac.AC_KERNEL_EPOCH, 64, 10, 0),
               ("blocked_lb32", ac.AC_KERNEL_BLOCKED, 32, 1, 8), ("blocked_lb64", ac.AC_KERNEL_BLOCKED, 64, 1, 8),
               ("blocked_lb128", ac.AC_KERNEL_BLOCKED, 128, 1, 8)]
    for name, kern, lb, rounds, polls in configs:
        with ac.Sim(w["rows"], w["cols"], 0.4407, w["J"], w["h"], seed, init=w["init"], kernel=kern, Lb=lb,
                    rounds=rounds, polls=polls) as s:
            s.run_until(w["T"])        # warm-up run
            s.reset(seed, w["init"])
            s.run_until(w["T"])
            st = s.stats()
        res[name] = {"events": st["events"], "device_ms": st["device_ms"],
                     "events_per_s": st["events"] / (st["device_ms"] / 1000.0),
                     "hbm_frac_effective": BYTES_PER_EVENT * st["events"] / (st["device_ms"] / 1000.0) / 1e9
                     / measured_peaks()[0],
                     "launches": st["launches"], "enabled_frac": st["enabled_frac_mean"],
                     "visits": st["visits"], "polls": st["polls"], "grid": st["grid"]}
    return res


if __name__ == "__main__":
    sys.exit(main())
