"""Benchmark of the GB300 aura exchange (classification, serialization,
difference encoding, byte packing, decoding) on a synthetic agent workload.

One step = one whole iteration of the exchange over every pair of one
population state.  States are generated on the device before timing (inputs
resident in HBM); each timed step consumes the next state of the series, so
the references chain exactly as in a simulation.  Every state (64 B/agent)
is far larger than L2, so no L2 flush is needed between steps.

Prints ONE JSON line (rank 0).  `--impl reference` times the CPU oracle on
the host cores instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "aura-exchange agents/s and encode+decode GB/s (% HBM peak); bytes/agent"

# Algorithmic bytes per launch of each kernel, from the totals of the launches:
# what each step must read and write.  N agents, E records, R reference slots,
# H placeholders, A new records, Y payload bytes.
def kernel_bytes(name, t):
    N, E, R, A, Y = t["agents"], t["records"], t["ref_slots"], t["new_records"], \
        t["payload_bytes"]
    M = E  # matched + new = records
    table = {
        "classify_kernel": 32 * N,
        "emit_kernel": 8 * N + 8 * E,
        "rs_hist_kernel": 4 * E,
        "rs_scatter_kernel": 16 * E,
        "pack_kernel": (4 + 64 + 64 + 16 + 4) * E,
        # record fields read and the record written per entry, its record
        # index; the mask of every agent
        "pack_runs_kernel": (64 + 64 + 4) * E + 4 * N,
        "enc_match_kernel": (64 + 16 + 4 + 4 + 4) * R + 64 * (R - t["holes"]),
        "enc_new_kernel": 4 * E + (64 + 16) * A,
        "enc_emit_kernel": 4 * R + 128 * (R - t["holes"]) + 4 * E + 64 * A + 4 * A + Y + 64 * M,
        "dec_sum_kernel": 4 * (R + A),
        "dec_emit_kernel": 4 * (R + A) + Y + 64 * (R - t["holes"]) + 64 * M,
        # the persistent kernel runs encode + decode: compulsory traffic only
        # (message, reference, new reference and wire on the sender; wire,
        # reference and receive buffers on the receiver)
        "codec_persistent_kernel": 64 * (3 * E + 2 * R) + 2 * t["wire_bytes"],
        # migration (N agents per step, L leavers): positions read to find the
        # owners; every record read and written once by the stable regroup;
        # leavers serialized (gather + arena write) and deserialized
        "mig_count_kernel": 24 * N,
        "mig_move_kernel": 128 * N + 8 * t.get("leavers", 0),
        "mig_pack_kernel": 128 * t.get("leavers", 0),
        "mig_unpack_kernel": 128 * t.get("leavers", 0),
    }
    return table.get(name)


# DRAM traffic of the dominant kernel per launch, from a one-pass ncu capture of
# the full-size run recorded in profiles/; used only while the kernel's sources
# are the ones the capture was taken with (their digest is recorded beside it).
KERNEL_SOURCES = {"codec_persistent_kernel": ("batched.cu", "codec.cuh", "tera_device.cuh"),
                  "mig_move_kernel": ("migrate.cu", "classify.cuh", "tera_device.cuh")}


def source_code_text(text: str) -> str:
    """The code of a C++/CUDA source without its comments and whitespace, so
    that the digest below changes with the code only (string literals kept)."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c == '"':
            j = i + 1
            while j < n and text[j] != '"':
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
        elif c.isspace():
            i += 1
        else:
            out.append(c)
            i += 1
    return "".join(out)


def kernel_digest(name):
    """Digest of the code (not the comments) of the sources a kernel is built from."""
    import hashlib
    files = KERNEL_SOURCES.get(name)
    if not files:
        return None
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2509_24063_gb300", "csrc", f), encoding="utf-8") as fh:
            h.update(source_code_text(fh.read()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(name, workload):
    """(bytes per launch, units per launch) recorded for this kernel and
    workload (units: records, or agents for migration kernels), or None when
    absent or taken with other kernel sources."""
    path = os.path.join(ROOT, "profiles", f"{name}_{workload}.md")
    try:
        with open(path) as f:
            text = f.read()
    except OSError:
        return None
    vals = {}
    for line in text.splitlines():
        if ":" in line and line.startswith("- "):
            k, v = line[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel source digest") != kernel_digest(name):
        return None
    units = vals.get("records per launch", vals.get("agents per launch"))
    try:
        return float(vals["DRAM bytes per launch"]), float(units)
    except (KeyError, TypeError, ValueError):
        return None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            sel = [] if self.gpu is None else [f"--id={self.gpu}"]
            self.proc = subprocess.Popen(
                ["nvidia-smi"] + sel + [f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append(dict(sm=float(f[1]), smax=float(f[2]), hw=f[5], hwt=f[6], swt=f[7],
                                 pcap=f[8]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        reasons = set()
        for r in rows:
            for k, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                            ("swt", "sw_thermal_slowdown"), ("pcap", "sw_power_cap")):
                if r[k].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in rows),
                "sm_max_mhz": max(r["smax"] for r in rows), "reasons": sorted(reasons),
                "samples": len(rows)}


def job_totals(elapsed_ms: float, agents: int, world: int, device) -> tuple:
    """Whole-job numbers of a replicated run: the slowest rank's time and the
    agents processed by all ranks."""
    if world <= 1:
        return elapsed_ms, agents
    import torch
    import torch.distributed as dist
    tt = torch.tensor([elapsed_ms], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    aa = torch.tensor([agents], device=device, dtype=torch.float64)
    dist.all_reduce(aa)
    return float(tt.item()), int(aa.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def cpu_sample_states(wl, states_gpu, n_sample):
    """First n_sample agents of two consecutive states, on the host."""
    from synth import to_numpy
    out = []
    for st in states_gpu:
        out.append(to_numpy({k: v[:n_sample] for k, v in st.items()}))
    return out


def host_cores():
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def oracle_time(wl, host_states, threads=1):
    """Oracle over a chain of host states (single-threaded, or with agents and
    pairs spread over `threads` host threads); returns per-state seconds."""
    import oracle
    g = oracle.make_grid(wl.lo, wl.hi, wl.grid, wl.w, wl.periodic)
    ref = recv_ref = None
    times = []
    for s in host_states:
        t0 = time.perf_counter()
        res = oracle.exchange_iteration(g, s, ref=ref, recv_ref=recv_ref, threads=threads)
        times.append(time.perf_counter() - t0)
        assert res["status"] == oracle.OK, res["status"]
        ref, recv_ref = (res["ref_next"], res["pair_off"]), (res["recv"], res["recv_off"])
    return times


def lz4_library():
    """liblz4 through its public C API, or None when the library is absent."""
    import ctypes as C
    for name in ("liblz4.so.1", "liblz4.so"):
        try:
            L = C.CDLL(name)
        except OSError:
            continue
        L.LZ4_compressBound.argtypes = [C.c_int]
        L.LZ4_compressBound.restype = C.c_int
        L.LZ4_compress_default.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int]
        L.LZ4_compress_default.restype = C.c_int
        return L
    return None


def compression_comparison(wl, host_states):
    """The paper's compression framing (Sec. 3.11) on the CPU sample, message
    by message: LZ4 alone on the raw TeraAgent IO buffers (header + records),
    LZ4 after the difference encoding (the XOR-serialized message of Sec. 2.3),
    and this codec's wire messages (header, codes, payload, padding)."""
    import numpy as np

    import oracle
    L = lz4_library()
    if L is None:
        return {"available": False, "reason": "liblz4 is not installed on this host"}

    def lz4_bytes(a):
        a = np.ascontiguousarray(a).view(np.uint8)
        n = int(a.nbytes)
        cap = L.LZ4_compressBound(n)
        out = np.empty(max(cap, 1), dtype=np.uint8)
        r = L.LZ4_compress_default(a.ctypes.data, out.ctypes.data, n, cap)
        assert r > 0 or n == 0
        return r

    g = oracle.make_grid(wl.lo, wl.hi, wl.grid, wl.w, wl.periodic)
    r0 = oracle.exchange_iteration(g, host_states[0])
    r1 = oracle.exchange_iteration(g, host_states[1], ref=(r0["ref_next"], r0["pair_off"]),
                                   recv_ref=(r0["recv"], r0["recv_off"]))
    assert r0["status"] == oracle.OK and r1["status"] == oracle.OK
    off0, off1 = r0["pair_off"], r1["pair_off"]
    raw = lz_raw = lz_delta = wire = msgs = 0
    for p in range(len(off1) - 1):
        m = int(off1[p + 1] - off1[p])
        if m == 0:
            continue
        a = (int(off1[p]) + p) * 64
        buf = r1["rec"][a:a + 64 * (m + 1)]  # header + records
        msg = buf[64:].view(np.uint64).reshape(-1, 8)
        ref = oracle.arena_pair(r0["ref_next"], off0, p)
        raw += buf.nbytes
        lz_raw += lz4_bytes(buf)
        lz_delta += lz4_bytes(oracle.delta_records(msg, ref))
        wire += int(r1["wire_len"][p])
        msgs += 1
    return {"available": True, "messages": msgs, "raw_bytes": raw, "lz4_bytes": lz_raw,
            "delta_lz4_bytes": lz_delta, "codec_bytes": wire,
            "raw_over_lz4": raw / lz_raw, "lz4_over_delta_lz4": lz_raw / lz_delta,
            "raw_over_codec": raw / wire,
            "sample": "second of two consecutive states of the CPU-baseline sample, every "
                      "non-empty message compressed on its own"}


def run_reference(args):
    """CPU oracle arm: W warm-up + K timed iterations on a bounded sample."""
    import torch
    from synth import WORKLOADS, Generator, scaled, to_numpy
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    wl0 = WORKLOADS[args.workload]
    n = min(wl0.n0, args.ref_agents)
    wl = scaled(wl0, n, boundary=args.boundary)
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    gen = Generator(wl, device=dev)
    states = [to_numpy(s) for s in gen.series(args.warmup + args.steps)]
    cores = host_cores()
    times = oracle_time(wl, states, threads=cores)
    timed = times[args.warmup:]
    agents = sum(int(s["x"].shape[0]) for s in states[args.warmup:])
    total = sum(timed)
    value = agents / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "agents/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": args.workload, "agents_per_step": n,
                   "note": f"oracle on the first {n} agents per state of the same workload"},
        "cpu_baseline": {"value": value, "unit": "agents/s", "cores": cores, "kind": "oracle",
                         "sample": f"{args.warmup}+{args.steps} iterations of {args.workload} "
                                   f"scaled to {n} agents (same cube, grid, aura, dynamics); "
                                   f"agents and pairs spread over {cores} host threads"},
        "e2e": {"value": value, "unit": "agents/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_migration(args):
    """Agent migration of a box-major state (one send + receive per step).

    The inputs are a chain of real transitions of the workload with its moves
    only (migration carries no births or deaths): the state after each
    migration, with the positions of the next iteration.  They are prepared
    before the timed region; each timed step migrates one of them."""
    import torch
    import torch.distributed as dist

    import paper_2509_24063_gb300 as tera
    from synth import WORKLOADS, Generator, scaled

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    wl = WORKLOADS[args.workload]
    if args.agents:
        wl = scaled(wl, args.agents)
    wl = dataclasses.replace(wl, p_grow=0.0, p_divide=0.0, p_die=0.0, boundary=args.boundary)
    total = args.warmup + args.steps
    gen = Generator(wl, device="cuda", seed=wl.seed + 7919 * rank)
    it = gen.series(total + 1)
    ctx = tera.Context(wl.lo, wl.hi, wl.grid, wl.w, device=local, periodic=wl.periodic)
    n = wl.n0
    # the regroup from box 0 moves nearly every agent: room for n leavers
    mig = tera.Migration(ctx, n, max_leavers=n)
    cur, off = mig.regroup(next(it))
    ctx.status()  # raises before any migrated id is used as an index
    inputs, leavers = [], []
    for _ in range(total):
        st = next(it)
        idx = cur["id"]  # move-only dynamics: agent id = index in the generated state
        moved = {k: (st[k][idx] if k in ("x", "y", "z") else cur[k]) for k in cur}
        del st
        nxt, off_next = mig.step(moved, off)
        ctx.status()
        leavers.append(int(mig.inbox_off[-1]))
        inputs.append((moved, off))
        cur, off = nxt, off_next
    del cur, off, gen, it
    ctx.status()
    out = mig.empty_like(inputs[0][0])
    off_out = torch.empty_like(inputs[0][1])
    for t in range(args.warmup):
        mig.step(inputs[t][0], inputs[t][1], out, off_out)
    ctx.status()
    ctx.profile_table(reset=True)
    ctx.profile(True)
    launches0 = ctx.launches
    stream = torch.cuda.current_stream()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(None if world == 1 else local) as clk:
        ev0.record(stream)
        for t in range(args.warmup, total):
            mig.step(inputs[t][0], inputs[t][1], out, off_out)
        ev1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    elapsed_ms = ev0.elapsed_time(ev1)
    launches = ctx.launches - launches0
    ctx.profile(False)
    prof = ctx.profile_table(reset=True)
    ctx.status()
    t_max, agents_all = job_totals(elapsed_ms, n * args.steps, world, "cuda")
    value = agents_all / (t_max / 1e3)
    lv = sum(leavers[args.warmup:])
    totals = {"agents": n * args.steps, "records": 0, "ref_slots": 0, "new_records": 0,
              "payload_bytes": 0, "holes": 0, "wire_bytes": 0, "leavers": lv}
    peaks, peak_kind = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    dname, (dn, dms) = max(prof.items(), key=lambda kv: kv[1][1])
    dbytes = kernel_bytes(dname, totals)
    roofline = None
    if dbytes is not None and dn > 0:
        achieved = dbytes / dn / (dms / dn / 1e3) / 1e9
        rec = recorded_traffic(dname, wl.name) if not args.agents else None
        traffic = rec[0] * n / rec[1] if rec is not None else None  # grows with the agents
        roofline = {"bound": "hbm", "kernel": dname, "achieved": achieved, "peak": hbm,
                    "unit": "GB/s", "frac": achieved / hbm, "traffic": traffic,
                    "peak_kind": peak_kind, "launches": dn, "avg_ms": dms / dn,
                    "algorithmic_bytes_per_launch": dbytes / dn}
    if args.profile_table and rank == 0:
        tot = sum(v[1] for v in prof.values())
        for k, (n_, ms_) in sorted(prof.items(), key=lambda kv: -kv[1][1]):
            b = kernel_bytes(k, totals)
            gbs = f"{b / (ms_ / 1e3) / 1e9:8.1f} GB/s" if b and ms_ > 0 else ""
            print(f"{k:24s} {n_:6d} launches {ms_:9.3f} ms {100 * ms_ / tot:5.1f}% {gbs}",
                  file=sys.stderr)
    del inputs, out, mig
    ctx.close()
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = migration_oracle_time(wl, min(args.cpu_sample, n))
    line = {
        "metric": "migration agents/s", "value": value, "unit": "agents/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic",
        "config": {"workload": wl.name + (f"@{args.agents}" if args.agents else ""),
                   "agents": n, "grid": list(wl.grid), "boundary": wl.boundary,
                   "dynamics": "moves only (p_move, step_sigma of the workload)",
                   "leavers_per_step": lv / args.steps,
                   "l2": "inputs larger than L2 (64 B/agent state per step)",
                   "parallelism": f"replicas{world}"},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": None,
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def migration_oracle_time(wl, ns):
    """Oracle migration step on a bounded sample: the workload scaled to ns
    agents (same cube, grid and moves), box-major, then moved once."""
    import numpy as np

    import oracle
    from synth import Generator, scaled, to_numpy
    w = scaled(wl, ns)
    g = oracle.make_grid(w.lo, w.hi, w.grid, w.w, w.periodic)
    states = [to_numpy(s) for s in Generator(w, device="cpu").series(2)]
    s0, s1 = states
    st, owner, _ = oracle.classify(g, s0["x"], s0["y"], s0["z"])
    perm = np.argsort(owner, kind="stable")
    nb = w.n_boxes
    off = np.zeros(nb + 1, dtype=np.uint64)
    off[1:] = np.cumsum(np.bincount(owner, minlength=nb))
    moved = {k: np.ascontiguousarray((s1 if k in ("x", "y", "z") else s0)[k][perm])
             for k in s0}
    t0 = time.perf_counter()
    res = oracle.migrate(g, moved, off)
    dt = time.perf_counter() - t0
    assert res["status"] == oracle.OK
    return {"value": ns / dt, "unit": "agents/s", "cores": 1, "kind": "oracle",
            "sample": f"one migration step of {wl.name} scaled to {ns} agents "
                      f"(same cube, grid, moves); single-threaded C oracle"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="tera", choices=["tera", "reference"])
    ap.add_argument("--workload", default="uniform_100m")
    ap.add_argument("--path", default="batched", choices=["batched", "all_pairs", "per_subdomain"])
    ap.add_argument("--no-graph", action="store_true", help="batched path without CUDA graphs")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--boundary", default="closed", choices=["closed", "toroidal"],
                    help="space boundary of the workload (toroidal: every axis wraps)")
    ap.add_argument("--ref-interval", type=int, default=1,
                    help="reference interval K (the reference is the message of every K-th iteration)")
    ap.add_argument("--tune", default="",
                    help="fixed batched schedule block,ctas_per_sm[,table_records] (skips the tuner)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-sample", type=int, default=2_000_000)
    ap.add_argument("--ref-agents", type=int, default=1_000_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--agents", type=int, default=0,
                    help="override the workload's agent count (profiling on a smaller case)")
    ap.add_argument("--profile-table", action="store_true", help="print per-kernel table to stderr")
    ap.add_argument("--predictor", action="store_true",
                    help="learned predictor: train on the workload's generated iterations, then "
                         "time and compare bytes/agent against plain XOR on fresh iterations")
    ap.add_argument("--migration", action="store_true",
                    help="agent migration of the box-major state instead of the aura exchange")
    ap.add_argument("--no-id-columns", action="store_true",
                    help="batched codec reads record ids from the records (no id columns)")
    ap.add_argument("--compare-paths", action="store_true",
                    help="agents/s of the per-subdomain, all-pairs and batched paths on the same "
                         "states (one JSON line)")
    ap.add_argument("--metrics-log", default="",
                    help="after the timed run, re-run its iterations eagerly and write one JSON "
                         "line per iteration to this file")
    ap.add_argument("--train-iters", type=int, default=200)
    ap.add_argument("--eval-iters", type=int, default=20)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "tera":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    if args.predictor:
        return run_predictor(args)
    if args.migration:
        return run_migration(args)
    if args.compare_paths:
        return run_compare_paths(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2509_24063_gb300 as tera
    from synth import WORKLOADS, Generator

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    wl = WORKLOADS[args.workload]
    if args.agents:
        from synth import scaled
        wl = scaled(wl, args.agents)
    if args.boundary != wl.boundary:
        wl = dataclasses.replace(wl, boundary=args.boundary)
    total_steps = args.warmup + args.steps
    # replicas: each rank runs its own seeded population (weak scaling, no exchange between ranks)
    gen = Generator(wl, device="cuda", seed=wl.seed + 7919 * rank)
    states = []
    for st in gen.series(total_steps):
        states.append({k: v for k, v in st.items() if k in
                       ("id", "x", "y", "z", "diameter", "volume", "adherence", "density")})
    del gen
    torch.cuda.synchronize()
    nmax = max(int(s["x"].shape[0]) for s in states)
    max_records = int(nmax * 0.35) + 4096 if wl.grid[0] >= 8 else 4 * nmax + 4096
    ctx = tera.Context(wl.lo, wl.hi, wl.grid, wl.w, device=local, periodic=wl.periodic)
    fixed = tuple(int(v) for v in args.tune.split(",")) if args.tune else None
    ex = tera.AuraExchange(ctx, max_agents=nmax, max_records=max_records, path=args.path,
                           tune=fixed, ref_interval=args.ref_interval,
                           id_columns=not args.no_id_columns)
    stream = torch.cuda.current_stream()
    use_graph = args.path == "batched" and not args.no_graph
    tune_info = {"tune": list(fixed), "candidates": 0} if fixed else None

    for t in range(args.warmup):
        if t == 1 and args.path == "batched" and not args.no_autotune and fixed is None:
            from paper_2509_24063_gb300 import autotune
            # tuned afresh on this workload (untimed warm-up), not from the cache
            tune, table = autotune.tune_batched(ex, states[t], use_cache=False)
            tune_info = {"tune": list(tune), "candidates": len(table)}
        else:
            ex.step(states[t])
    ctx.status()  # raises on any device-side error
    ctx.stats(reset=True)
    ctx.profile_table(reset=True)
    ctx.profile(True)
    launches0 = ctx.launches
    graphs = None
    if use_graph:
        graphs = [ex.capture(states[t], t) for t in range(args.warmup, total_steps)]
    launches_captured = ctx.launches - launches0

    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(None if world == 1 else local) as clk:
        ev0.record(stream)
        for t in range(args.warmup, total_steps):
            if graphs is not None:
                graphs[t - args.warmup].replay()
                ex.advance()
            else:
                ex.step(states[t])
        ev1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    elapsed_ms = ev0.elapsed_time(ev1)
    launches = launches_captured if graphs is not None else ctx.launches - launches0
    del graphs
    ctx.profile(False)
    prof = ctx.profile_table(reset=True)
    stats = ctx.stats(reset=True)
    ctx.status()
    agents = sum(int(states[t]["x"].shape[0]) for t in range(args.warmup, total_steps))
    t_max, agents_all = job_totals(elapsed_ms, agents, world, "cuda")
    value = agents_all / (t_max / 1e3)

    # encode+decode algorithmic bytes over the timed steps (pack .. decode)
    codec_kernels = ("pack_kernel", "enc_match_kernel", "enc_new_kernel", "enc_emit_kernel",
                     "dec_sum_kernel", "dec_emit_kernel")
    H = stats["holes"]
    R, E, A, Y = stats["ref_slots"], stats["records"], stats["new_records"], \
        stats["payload_bytes"]
    codec_bytes = kernel_bytes("pack_kernel", stats) + kernel_bytes("codec_persistent_kernel", stats)
    codec_ms = sum(prof.get(k, (0, 0.0))[1] for k in prof
                   if k.startswith(("pack", "enc_", "dec_", "bat_", "codec_", "unit_map")))
    peaks, peak_kind = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    codec_gbs = codec_bytes / (codec_ms / 1e3) / 1e9 if codec_ms > 0 else None

    # dominant kernel
    dname, (dn, dms) = max(prof.items(), key=lambda kv: kv[1][1]) if prof else ("", (0, 0.0))
    dbytes = kernel_bytes(dname, stats)
    roofline = None
    if dbytes is not None and dn > 0:
        per_launch_bytes = dbytes / dn
        per_launch_s = dms / dn / 1e3
        achieved = per_launch_bytes / per_launch_s / 1e9
        rec = recorded_traffic(dname, wl.name) if not args.agents else None
        traffic = None
        if rec is not None:
            # scaled to this run's records per launch (traffic grows with them)
            traffic = rec[0] * (stats["records"] / dn) / rec[1]
        roofline = {"bound": "hbm", "kernel": dname, "achieved": achieved, "peak": hbm,
                    "unit": "GB/s", "frac": achieved / hbm, "traffic": traffic,
                    "peak_kind": peak_kind, "launches": dn, "avg_ms": dms / dn,
                    "algorithmic_bytes_per_launch": per_launch_bytes}
    if args.profile_table and rank == 0:
        tot = sum(v[1] for v in prof.values())
        for k, (n_, ms_) in sorted(prof.items(), key=lambda kv: -kv[1][1]):
            b = kernel_bytes(k, stats)
            gbs = f"{b / (ms_ / 1e3) / 1e9:8.1f} GB/s" if b and ms_ > 0 else ""
            print(f"{k:24s} {n_:6d} launches {ms_:9.3f} ms {100 * ms_ / tot:5.1f}% {gbs}",
                  file=sys.stderr)
        print(json.dumps(stats), file=sys.stderr)

    # per-iteration metrics: the same iterations again, eager, untimed by the line above
    metrics_rows = []
    if args.metrics_log and rank == 0:
        ex.reset()
        ctx.stats(reset=True)
        ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for t in range(total_steps):
            ea.record(stream)
            ex.step(states[t])
            eb.record(stream)
            torch.cuda.synchronize()
            st = ctx.stats(reset=True)
            ms = ea.elapsed_time(eb)
            n = int(states[t]["x"].shape[0])
            step_bytes = kernel_bytes("pack_kernel", st) + kernel_bytes("codec_persistent_kernel", st)
            metrics_rows.append({
                "workload": args.workload + (f"@{args.agents}" if args.agents else ""),
                "path": args.path, "tune": list(ex.tune) if ex.tune else None,
                "ref_interval": args.ref_interval, "iteration": t, "agents": n,
                "pairs": ctx.n_pairs, "aura_records": st["records"], "ref_slots": st["ref_slots"],
                "new_records": st["new_records"], "holes": st["holes"],
                "raw_bytes": 64 * st["records"], "packed_bytes": st["wire_bytes"],
                "payload_bytes": st["payload_bytes"], "ms_eager": ms,
                "agents_per_s": n / (ms / 1e3),
                "pack_codec_gbs": step_bytes / (ms / 1e3) / 1e9,
                "pack_codec_hbm_frac": step_bytes / (ms / 1e3) / 1e9 / hbm})
        ctx.status()

    # the CPU baseline's sample (host copies) and the end-to-end inputs are
    # taken from the device states; then every device buffer of the measured
    # run is released, so the end-to-end leg runs on a clean device
    hs = None
    ns = 0
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ns = min(args.cpu_sample, int(states[0]["x"].shape[0]))
        hs = cpu_sample_states(wl, states[args.warmup - 1:args.warmup + 1], ns)
    agents_cfg = int(states[args.warmup]["x"].shape[0])
    tune_e2e = ex.tune
    ex_id_columns = ex.id_columns
    e2e_host = None
    if args.e2e_steps > 0:
        e2e_host = e2e_inputs(args, states)
    del ex, states
    ctx.close()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()

    # end to end: host-resident state in, wire messages out, through the same API
    e2e = None
    if e2e_host is not None:
        e2e = run_e2e(args, tera, wl, e2e_host, nmax, max_records, local, tune_e2e)
        del e2e_host

    cpu = compression = None
    if hs is not None:
        from synth import scaled
        cores = host_cores()
        tms1 = oracle_time(scaled(wl, ns), hs)
        tmsn = oracle_time(scaled(wl, ns), hs, threads=cores)
        compression = compression_comparison(scaled(wl, ns), hs)
        na = int(hs[1]["x"].shape[0])
        cpu = {"value": na / tmsn[1], "unit": "agents/s", "cores": cores,
               "kind": "oracle",
               "sample": f"one iteration (with reference) of the first {ns} agents of two "
                         f"consecutive states of {args.workload}; C oracle with agents and pairs "
                         f"spread over {cores} host threads",
               "single_core": {"value": na / tms1[1], "unit": "agents/s", "cores": 1}}
    if metrics_rows:
        with open(args.metrics_log, "w") as f:
            for row in metrics_rows:
                row["host_cores"] = host_cores()
                if cpu is not None:
                    row["oracle_agents_per_s"] = cpu["value"]
                    row["oracle_ms_per_iteration"] = row["agents"] / cpu["value"] * 1e3
                f.write(json.dumps(row) + "\n")
    clk_sum = clk.summary()
    line = {
        "metric": METRIC, "value": value, "unit": "agents/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic",
        "config": {"workload": args.workload + (f"@{args.agents}" if args.agents else ""),
                   "agents": agents_cfg,
                   "grid": list(wl.grid), "aura_width": wl.w, "path": args.path,
                   "cuda_graph": use_graph, "tune": tune_info, "ref_interval": args.ref_interval,
                   "id_columns": bool(ex_id_columns),
                   "boundary": wl.boundary,
                   "l2": "inputs larger than L2 (64 B/agent state per step)",
                   "parallelism": f"replicas{world}"},
        "encode_decode_gbs": codec_gbs,
        "encode_decode_hbm_frac": (codec_gbs / hbm) if codec_gbs else None,
        "bytes_per_agent": stats["wire_bytes"] / max(1, E),
        "records_per_step": E / args.steps,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "compression": compression,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk_sum,
    }
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_predictor(args):
    """Train the predictor on the workload's generated iterations (seed A),
    then run fresh iterations (seed B) with and without it: agents/s of the
    predictor path (timed, states resident) and wire bytes per record of both."""
    import torch
    import paper_2509_24063_gb300 as tera
    from paper_2509_24063_gb300 import predictor
    from synth import WORKLOADS, Generator, scaled
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    wl = WORKLOADS["drift_16m" if args.workload == "uniform_100m" else args.workload]
    if args.agents:
        wl = scaled(wl, args.agents)
    t0 = time.time()
    gen = Generator(wl, device="cuda")
    nmax = int(wl.n0 * 1.05) + 4096
    max_records = 2 * nmax
    ctx = tera.Context(wl.lo, wl.hi, wl.grid, wl.w, device=local, periodic=wl.periodic)
    ex = tera.AuraExchange(ctx, nmax, max_records, path="all_pairs", predictor=True)
    every = max(1, args.train_iters // 20)
    picks = set(range(2, args.train_iters, every))
    per = max_records * 12
    samples = torch.zeros(len(picks) * per, dtype=torch.float32, device="cuda")
    k = 0
    for t, st in enumerate(gen.series(args.train_iters)):
        if t in picks:
            ex.samples = samples[k * per:(k + 1) * per]
            k += 1
        else:
            ex.samples = None
        ex.step({f: st[f] for f in ("id", "x", "y", "z", "diameter", "volume", "adherence",
                                     "density")})
    ctx.status()
    del ex
    params = predictor.init_params(5)
    t1 = time.time()
    nv = predictor.train(ctx, samples, params)
    torch.cuda.synchronize()
    t2 = time.time()
    del samples
    evals = [{f: st[f] for f in ("id", "x", "y", "z", "diameter", "volume", "adherence",
                                   "density")}
             for st in Generator(wl, device="cuda", seed=wl.seed + 1).series(args.eval_iters)]
    skip = min(3, len(evals) - 1)
    bx, rx = predictor.wire_bytes(ctx, evals, nmax, max_records, skip=skip)
    ex = tera.AuraExchange(ctx, nmax, max_records, path="batched", params=params)
    for t in range(skip):
        ex.step(evals[t])
    ctx.status()
    ctx.stats(reset=True)
    ctx.profile_table(reset=True)
    ctx.profile(True)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(None) as clk:
        e0.record(stream)
        for t in range(skip, len(evals)):
            ex.step(evals[t])
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    ctx.profile(False)
    prof = ctx.profile_table(reset=True)
    if args.profile_table:
        tot = sum(v[1] for v in prof.values())
        for k, (n_, ms_) in sorted(prof.items(), key=lambda kv: -kv[1][1]):
            print(f"{k:24s} {n_:6d} launches {ms_:9.3f} ms {100 * ms_ / tot:5.1f}%",
                  file=sys.stderr)
    st = ctx.stats(reset=True)
    ctx.status()
    del ex
    # the same iterations on the plain batched path (XOR difference only), also eager
    ex = tera.AuraExchange(ctx, nmax, max_records, path="batched")
    for t in range(skip):
        ex.step(evals[t])
    ctx.status()
    torch.cuda.synchronize()
    e0.record(stream)
    for t in range(skip, len(evals)):
        ex.step(evals[t])
    e1.record(stream)
    torch.cuda.synchronize()
    ms_xor = e0.elapsed_time(e1)
    ctx.status()
    del ex
    steps = len(evals) - skip
    agents = sum(int(evals[t]["x"].shape[0]) for t in range(skip, len(evals)))
    line = {
        "metric": METRIC, "value": agents / (ms / 1e3), "unit": "agents/s", "n_gpus": 1,
        "steps": steps, "warmup": skip, "ms_per_step": ms / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64+f32", "data": "synthetic",
        "config": {"workload": wl.name + (f"@{args.agents}" if args.agents else ""),
                   "agents": int(evals[-1]["x"].shape[0]), "train_iterations": args.train_iters,
                   "eval_iterations": args.eval_iters, "path": "batched+predictor"},
        "bytes_per_agent_xor": bx / max(1, rx),
        "bytes_per_agent_residual": st["wire_bytes"] / max(1, st["records"]),
        "residual_vs_xor": (st["wire_bytes"] / max(1, st["records"])) / (bx / max(1, rx)),
        "records_per_step": st["records"] / max(1, steps),
        "ref_slots_per_step": st["ref_slots"] / max(1, steps),
        "xor_ms_per_step": ms_xor / steps,
        "predictor_vs_xor_time": ms / max(ms_xor, 1e-9),
        "training": {"samples": nv, "steps": 4000, "batch": 8192, "lr": 0.02, "clip": 1.0,
                     "seconds": t2 - t1, "collect_seconds": t1 - t0},
        "clocks": clk.summary(),
    }
    print(json.dumps(line))
    ctx.close()
    return 0


def run_compare_paths(args):
    """The three paths of the exchange on the same states: one launch per
    sending box (per_subdomain), one launch per step for all pairs
    (all_pairs), and the persistent batched codec replayed from CUDA graphs
    (batched, schedule tuned at warm-up).  Each path runs W warm-up and K timed
    iterations of the same chain; the bytes produced are the same on every
    path (the parity tests check it), so only the time differs."""
    import torch

    import paper_2509_24063_gb300 as tera
    from paper_2509_24063_gb300 import autotune
    from synth import WORKLOADS, Generator, scaled
    wl = WORKLOADS[args.workload]
    if args.agents:
        wl = scaled(wl, args.agents)
    total = args.warmup + args.steps
    states = [{k: v for k, v in st.items() if k in
               ("id", "x", "y", "z", "diameter", "volume", "adherence", "density")}
              for st in Generator(wl, device="cuda").series(total)]
    nmax = max(int(s["x"].shape[0]) for s in states)
    max_records = int(nmax * 0.35) + 4096 if wl.grid[0] >= 8 else 4 * nmax + 4096
    out = {}
    stream = torch.cuda.current_stream()
    with ClockSampler(None) as clk:
        for path in ("per_subdomain", "all_pairs", "batched"):
            ctx = tera.Context(wl.lo, wl.hi, wl.grid, wl.w, periodic=wl.periodic)
            ex = tera.AuraExchange(ctx, max_agents=nmax, max_records=max_records, path=path)
            for t in range(args.warmup):
                if t == 1 and path == "batched":
                    autotune.tune_batched(ex, states[t], use_cache=False)
                else:
                    ex.step(states[t])
            ctx.status()
            graphs = None
            if path == "batched":
                graphs = [ex.capture(states[t], t) for t in range(args.warmup, total)]
            launches0 = ctx.launches
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for t in range(args.warmup, total):
                if graphs is not None:
                    graphs[t - args.warmup].replay()
                    ex.advance()
                else:
                    ex.step(states[t])
            e1.record(stream)
            torch.cuda.synchronize()
            ctx.status()
            ms = e0.elapsed_time(e1)
            agents = sum(int(states[t]["x"].shape[0]) for t in range(args.warmup, total))
            out[path] = {"agents_per_s": agents / (ms / 1e3), "ms_per_step": ms / args.steps,
                         "launches_per_step": None if graphs is not None else
                         (ctx.launches - launches0) / args.steps,
                         "cuda_graph": graphs is not None}
            del graphs, ex
            ctx.close()
            torch.cuda.synchronize()
            torch.cuda.empty_cache()
    base = out["per_subdomain"]["agents_per_s"]
    line = {"metric": "aura-exchange agents/s by path", "unit": "agents/s",
            "workload": wl.name + (f"@{args.agents}" if args.agents else ""),
            "agents": int(states[args.warmup]["x"].shape[0]), "steps": args.steps,
            "warmup": args.warmup, "paths": out,
            "batched_over_per_subdomain": out["batched"]["agents_per_s"] / base,
            "all_pairs_over_per_subdomain": out["all_pairs"]["agents_per_s"] / base,
            "clocks": clk.summary()}
    print(json.dumps(line))
    return 0


def e2e_inputs(args, states):
    """Pinned host copies of the states the end-to-end leg runs on (the one
    before the timed ones, then e2e_steps timed ones)."""
    from paper_2509_24063_gb300.host import FIELDS
    k = min(args.e2e_steps, args.steps)
    return [{f: states[t][f].cpu().pin_memory() for f in FIELDS}
            for t in range(args.warmup - 1, args.warmup + k)]


def run_e2e(args, tera, wl, host, nmax, max_records, local, tune=None):
    """Same metric through the public API on host-resident state
    (paper_2509_24063_gb300.host.HostExchange): every step copies the eight
    state columns from pinned host memory and writes the used wire bytes back
    into pinned host memory; the next step's inputs are copied while a step
    computes (double-buffered device inputs)."""
    import torch
    from paper_2509_24063_gb300.host import FIELDS, HostExchange
    k = len(host) - 1
    ctx = tera.Context(wl.lo, wl.hi, wl.grid, wl.w, device=local, periodic=wl.periodic)
    hx = HostExchange(ctx, nmax, max_records, path=args.path, tune=tune,
                      ref_interval=args.ref_interval)
    outs = [torch.empty(hx.wire_capacity, dtype=torch.uint8).pin_memory() for _ in range(2)]
    hx.step(host[0], outs[0]).wait()  # first iteration of this chain (allocates scratch)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pend = [hx.step(hs, outs[(i + 1) % 2]) for i, hs in enumerate(host[1:])]
    nbytes = [p.wait() for p in pend]
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    agents = sum(int(hs["x"].shape[0]) for hs in host[1:])
    h2d = sum(int(hs[f].numel() * hs[f].element_size()) for hs in host[1:] for f in FIELDS)
    ctx.status()
    # the host link's own rate for one step's input copies (pinned host to
    # device, the same columns into the same device buffers, nothing else
    # running): the bound the end-to-end number is read against
    hs, buf = host[1], hx.inputs[0]
    n1 = int(hs["x"].shape[0])
    copy = torch.cuda.Stream(device=local)
    l0, l1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(copy):
        for f in FIELDS:
            buf[f][:n1].copy_(hs[f], non_blocking=True)
        l0.record(copy)
        for _ in range(3):
            for f in FIELDS:
                buf[f][:n1].copy_(hs[f], non_blocking=True)
        l1.record(copy)
    l1.synchronize()
    step_bytes = sum(int(hs[f].numel() * hs[f].element_size()) for f in FIELDS)
    link_gbs = 3 * step_bytes / (l0.elapsed_time(l1) / 1e3) / 1e9
    ctx.close()
    return {"value": agents / dt, "unit": "agents/s", "h2d_bytes_per_step": h2d // k,
            "d2h_bytes_per_step": sum(nbytes) // k, "steps": k,
            "overlap": "inputs of step t+1 copied while step t computes",
            "h2d_link_gbs": link_gbs,
            "link_bound_agents_per_s": n1 / (step_bytes / (link_gbs * 1e9))}


if __name__ == "__main__":
    sys.exit(main())
