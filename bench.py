"""Benchmark of the device-resident decode path.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload fastq|tiny|batch|genome] [options]

fastq (default): whole-file decode of the 1 GiB interleaved paired-end FASTQ
  workload (16 KiB blocks): decompressed GB/s, the decode kernel's fraction of
  the HBM roofline, random-read p50/p99 latency through the read-to-block
  index, an end-to-end figure through the C ABI with host buffers, and the CPU
  oracle decoder timed on this host.
tiny: the 2,000-read FASTQ (L2-resident): decode latency and read-lookup
  p50/p99 for every read.
batch: 4,096 FASTQ archives of log-uniform size (16 KiB-16 MiB) in one
  persistent launch replayed from a CUDA graph (autotuned launch shape),
  against one launch per archive.
genome: FASTA genome (50 GB by default) streamed through a 4 GiB device ring
  with a CRC-32 per window, then random 150-byte region lookups p50/p99.

One JSON line on rank 0. Whole-file decode does not shard; multi-GPU runs
(torchrun) decode one replica per GPU and report the aggregate.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time
import zlib
from concurrent.futures import ThreadPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "decompressed GB/s device-resident"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="fastq", choices=["fastq", "tiny", "batch", "genome", "serve", "entropy", "fastq_streams",
                                                         "encode"])
    p.add_argument("--log2-block", type=int, default=14)
    p.add_argument("--size", type=int, default=0, help="workload bytes (0 = the workload's default)")
    p.add_argument("--min-match", type=int, default=0, help="0 = the workload's default")
    p.add_argument("--reads", type=int, default=200, help="random reads timed (fastq)")
    p.add_argument("--max-level", type=int, default=8, help="fastq: the encoder's dependency-level cap")
    p.add_argument("--batch-count", type=int, default=4096)
    p.add_argument("--batch-max", type=int, default=1 << 24)
    p.add_argument("--ring", type=int, default=4 << 30)
    p.add_argument("--window", type=int, default=2 << 30)
    p.add_argument("--regions", type=int, default=100_000)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--encode-input", default="fastq", choices=["fastq", "fasta"],
                   help="encode: the paired-end FASTQ (1 GiB) or the FASTA genome generator (2 GB, D = 1 GiB)")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-tune", action="store_true")
    p.add_argument("--rates", default="1000,10000,100000", help="serve: arrival rates per second")
    p.add_argument("--requests", type=int, default=3000, help="serve: requests per rate")
    p.add_argument("--budget", type=int, default=8 << 30, help="serve: device-memory budget")
    p.add_argument("--slots", type=int, default=4, help="serve: batches in flight")
    p.add_argument("--no-phases", action="store_true", help="fastq: skip the per-phase split leg")
    p.add_argument("--no-side", action="store_true", help="fastq: skip the bounded batch and serving legs")
    p.add_argument("--phase-child", default="", help=argparse.SUPPRESS)
    return p.parse_args()


def recorded_traffic(key):
    """DRAM bytes per launch recorded from an ncu capture (profiles/traffic.json),
    or None when the kernel source changed since the capture."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
        src = os.path.join(ROOT, "paper_2606_18900_gb300", "csrc", "kernels.cu")
        if hashlib.sha256(open(src, "rb").read()).hexdigest() != rec["kernels_cu_sha256"]:
            return None
        return rec[key]["traffic_bytes"]
    except Exception:
        return None


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampler (100 ms period) around a region of sustained load."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, pw, reasons = [], 0.0, [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx = max(mx, float(f[2]))
                    pw.append(float(f[3]))
                except ValueError:
                    continue
                for n, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
            os.unlink(self.path)
        except Exception:
            pass
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm),
                "power_w_median": float(np.median(pw)) if pw else None}


def sustain(fn, seconds):
    """Keep the GPU busy with fn() for about `seconds` (for the clock sampler)."""
    import torch
    t = time.perf_counter()
    while time.perf_counter() - t < seconds:
        for _ in range(8):
            fn()
        torch.cuda.synchronize()


def timed_steps(fn, stream, steps):
    """Per-step CUDA-event times (ms) of fn() on stream."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        ev[i][0].record(stream)
        fn()
        ev[i][1].record(stream)
    stream.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def pctl(xs, q):
    return float(np.percentile(np.asarray(xs, dtype=np.float64), q)) if len(xs) else None


def base_line(args, value, ms_per_step, world, config, **extra):
    line = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8", "data": "synthetic", "config": config}
    line.update(extra)
    return line


def cpu_oracle_baseline(arc, data, what):
    """The CPU oracle decoder as it stands (single thread) on the given archive,
    and, beside it, the oracle's segment decoder run level by level on every
    host core (the all-core baseline)."""
    import oracle

    t = time.perf_counter()
    out = oracle.decode(arc)
    dt = time.perf_counter() - t
    cores = len(os.sched_getaffinity(0))
    t = time.perf_counter()
    out2 = oracle.decode_wavefront(arc, cores)
    dt2 = time.perf_counter() - t
    return {"value": data.size / dt / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": f"{what}: one sequential pass over {data.size} bytes ({dt:.1f} s); host has {cores} cores",
            "bit_exact": bool(np.array_equal(out, data)),
            "all_cores": {"value": data.size / dt2 / 1e9, "unit": "GB/s", "cores": cores,
                          "kind": "oracle segment decoder, level-by-level wavefront on all host cores",
                          "bit_exact": bool(np.array_equal(out2, data))}}


# ------------------------------------------------------------------- fastq

def shared_archive(make, path, rank, world):
    """Rank 0 runs make() (the encoder) once and publishes the archive at
    `path`; the other ranks wait at a barrier and read it. Returns (archive,
    seconds rank 0 spent in make)."""
    if world > 1 and rank != 0:
        import torch.distributed as dist
        dist.barrier()
        return np.fromfile(path, dtype=np.uint8), 0.0
    t = time.perf_counter()
    arc = make()
    dt = time.perf_counter() - t
    if world > 1:
        import torch.distributed as dist
        arc.tofile(path + ".tmp")
        os.replace(path + ".tmp", path)
        dist.barrier()
    return arc, dt


def max_over_ranks(value, world, device="cpu"):
    """The slowest rank's time: all-reduce MAX (identity for one rank)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_fastq(size, log2_block, min_match, rank, world, max_level=8):
    """The paired-end FASTQ workload encoded by the library encoder; with
    several ranks, one replica shared through /dev/shm."""
    import paper_2606_18900_gb300 as ace
    import synth

    data = synth.pe_fastq(size)
    path = f"/dev/shm/aceapex_bench_{size}_{log2_block}_{min_match}_{max_level}.bin"
    arc, enc_s = shared_archive(
        lambda: ace.encode(data, log2_B=log2_block, min_match=min_match, max_level=max_level,
                           reads=ace.fastq_index(data)), path, rank, world)
    return data, arc, enc_s


def random_reads(arc, data, n, seed, stream, device):
    """Per-read latency (ms) of read lookup + range decode, synchronous."""
    import torch
    import synth

    n_reads = arc.stats()["n_reads"]
    ids = synth.uniform(seed, 7, n, n_reads)
    buf = torch.empty(1 << 16, dtype=torch.uint8, device=device)
    lat, ok, segs, levels = [], True, [], []
    for k, r in enumerate(ids):
        torch.cuda.synchronize()
        t = time.perf_counter()
        lo, hi = arc.read_lookup(int(r))
        arc.decode_range(lo, hi, buf, stream)
        stream.synchronize()
        lat.append((time.perf_counter() - t) * 1e3)
        if k < 32:
            ok &= bytes(buf[: hi - lo].cpu().numpy()) == data[lo:hi].tobytes()
        nseg, lv = arc.range_closure(lo, hi)
        segs.append(nseg)
        levels.append(lv)
    arc.check(stream)
    closure = {"what": "segments decoded per read (the read's segments and their transitive sources) and the "
                       "wavefront depth (deepest level + 1)",
               "segments_p50": pctl(segs, 50), "segments_p99": pctl(segs, 99), "segments_max": max(segs) if segs else None,
               "depth_p50": pctl([v + 1 for v in levels], 50), "depth_max": max(levels) + 1 if levels else None}
    return lat, ok, closure


def level_cap_leg(data, args, min_match, stream, local, ratio):
    """The same data encoded with the dependency-level cap at 2 instead of 8:
    its ratio, whole-file decode rate and random reads (the cap bounds the
    wavefront depth of every read's closure at 3, at a ratio cost)."""
    import torch

    import paper_2606_18900_gb300 as ace

    t = time.perf_counter()
    arc_bytes = ace.encode(data, log2_B=args.log2_block, min_match=min_match, max_level=2,
                           reads=ace.fastq_index(data))
    enc_s = time.perf_counter() - t
    with ace.Archive(arc_bytes, device=local) as arc:
        out = torch.empty(data.size, dtype=torch.uint8, device=f"cuda:{local}")
        run = lambda: arc.decode_all(out, stream)
        for _ in range(args.warmup):
            run()
        arc.check(stream)
        ok = bool(np.array_equal(out.cpu().numpy(), data))
        step_ms = timed_steps(run, stream, args.steps)
        arc.check(stream)
        del out
        lat, reads_ok, closure = (random_reads(arc, data, args.reads, 2, stream, f"cuda:{local}") if args.reads
                                  else ([], True, None))
    ms = float(np.mean(step_ms))
    return {"what": "the workload's data encoded with the dependency-level cap 2 (the line's archive: cap 8)",
            "ratio": round(data.size / arc_bytes.size, 3), "ratio_cap_8": round(ratio, 3),
            "ms_per_step": ms, "gbs": data.size / (ms * 1e-3) / 1e9,
            "random_read": {"p50_ms": pctl(lat, 50), "p99_ms": pctl(lat, 99), "n": len(lat), "closure": closure},
            "encode_seconds": round(enc_s, 1), "bit_exact": ok and reads_ok}


PHASES = ("cmd_rans", "parse", "lit_rans", "src_checks", "copies", "loop", "dep_waits")
COUNTS = ("chunks", "rounds", "units", "segments", "waited_chunks")


def phase_child(args):
    """Runs under ACEAPEX_LIBRARY=phases (the library build with per-phase
    cycle counters): decodes the archive in args.phase_child and prints the
    warp-cycle share of every phase of the decode kernel and its event
    counts."""
    import ctypes
    import torch

    import paper_2606_18900_gb300 as ace

    arc_bytes = np.fromfile(args.phase_child, dtype=np.uint8)
    L = ace.lib()
    L.aceapex_phase_cycles.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
    L.aceapex_phase_cycles.restype = ctypes.c_int
    buf = (ctypes.c_uint64 * 12)()
    with ace.Archive(arc_bytes) as a:
        out = torch.empty(a.size, dtype=torch.uint8, device="cuda")
        stream = torch.cuda.Stream()
        for _ in range(2):
            a.decode_all(out, stream)
        a.check(stream)
        if L.aceapex_phase_cycles(buf, 12, 1):
            raise SystemExit("phase counters unavailable")
        reps = 5
        for _ in range(reps):
            a.decode_all(out, stream)
        a.check(stream)
        if L.aceapex_phase_cycles(buf, 12, 1):
            raise SystemExit("phase counters unavailable")
    cyc = [int(v) for v in buf[:6]] + [int(buf[11])]
    tot = sum(cyc)
    print(json.dumps({"share": {k: v / tot for k, v in zip(PHASES, cyc)},
                      "per_decode": {k: int(v) // reps for k, v in zip(COUNTS, buf[6:11])}}), flush=True)


def phase_split(arc_bytes, ms_decode, U):
    """Warp-time split of the decode kernel between its entropy phases
    (command-class rANS, command parse, literal rANS and placement) and its
    match phases (dependency waits, match copies), measured by the library
    build with per-phase cycle counters in a child process, applied to the
    plain build's kernel time."""
    path = f"/dev/shm/aceapex_phase_{os.getpid()}.bin"
    arc_bytes.tofile(path)
    try:
        env = dict(os.environ, ACEAPEX_LIBRARY="phases")
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--phase-child", path], env=env,
                           capture_output=True, text=True, timeout=600)
    finally:
        os.unlink(path)
    if r.returncode != 0:
        return {"error": (r.stderr or r.stdout).strip()[-300:]}
    j = json.loads(r.stdout.strip().splitlines()[-1])
    sh = j["share"]
    ent = sh["cmd_rans"] + sh["parse"] + sh["lit_rans"]
    mat = sh["src_checks"] + sh["copies"] + sh["dep_waits"]
    return {"what": "share of the decode kernel's warp cycles per phase (clock64 counters in a separate build), "
                    "applied to the plain build's median kernel time",
            "entropy_ms": ent * ms_decode, "match_ms": mat * ms_decode, "other_ms": sh["loop"] * ms_decode,
            "entropy_gbs_if_alone": U / (ent * ms_decode * 1e-3) / 1e9 if ent else None,
            "match_gbs_if_alone": U / (mat * ms_decode * 1e-3) / 1e9 if mat else None,
            "share": {k: round(v, 4) for k, v in sh.items()}, "events_per_decode": j["per_decode"]}


def workload_fastq(args):
    import torch

    import paper_2606_18900_gb300 as ace

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    size = args.size or (1 << 30)
    min_match = args.min_match or 16
    data, arc_bytes, enc_s = make_fastq(size, args.log2_block, min_match, rank, world, args.max_level)
    N = data.size
    arc = ace.Archive(arc_bytes, device=local)
    st = arc.stats()
    C, U, M = st["compressed_bytes"], st["decoded_bytes"], st["match_bytes"]
    out = torch.empty(N, dtype=torch.uint8, device=f"cuda:{local}")
    stream = torch.cuda.Stream()
    run = lambda: arc.decode_all(out, stream)

    for _ in range(args.warmup):
        run()
    arc.check(stream)
    ok = bool(np.array_equal(out.cpu().numpy(), data))
    if not ok:
        raise SystemExit("bench: GPU output differs from the input")

    clocks = Clocks(local)
    clocks.start()
    sustain(run, 0.4)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    step_ms = timed_steps(run, stream, args.steps)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    sustain(run, 0.4)
    clk = clocks.stop()
    arc.check(stream)
    total_ms = max_over_ranks(float(sum(step_ms)), world, f"cuda:{local}")
    value = N * world * args.steps / (total_ms * 1e-3) / 1e9
    avg_ms = float(np.mean(step_ms))
    peak, peak_kind = read_peaks()
    achieved = (C + U + M) / (avg_ms * 1e-3) / 1e9

    lat, reads_ok, closure = (random_reads(arc, data, args.reads, 2, stream, f"cuda:{local}") if args.reads
                              else ([], True, None))
    phases = None
    if rank == 0 and not args.no_phases:
        phases = phase_split(arc_bytes, float(np.median(step_ms)), U)
    batch = serve = None
    if rank == 0 and not args.no_side:
        # bounded samples of the batch and serving configurations, so that the
        # default line carries the batched-vs-plain and served-vs-serial
        # comparisons (the full-size runs: --workload batch / serve)
        batch = batch_compare(512, 2 << 20, 10, tune=False)
        batch["what"] = ("512 log-uniform 16 KiB-2 MiB FASTQ archives: one graph-replayed persistent launch against "
                         "one decode call per archive")
        serve = serve_compare(256_000_000, [100_000.0], 20_000, 4 << 30, 4, serial_n=300)
        serve["what"] = ("2,000-read FASTQ + 256 MB genome, 20,000 requests offered at 100k/s from the library's "
                         "submitting thread, against serial per-request decode")
    level_cap = None
    if rank == 0 and not args.no_side and args.max_level != 2:
        level_cap = level_cap_leg(data, args, min_match, stream, local, ratio=N / arc_bytes.size)

    # end to end through the C ABI with host buffers, every step: the archive
    # from pinned host memory to the output in pinned host memory by one
    # aceapex_decode_host call (open with the payload uploaded in pieces that
    # the window decodes overtake, windows copied out while the next ones
    # decode, close); beside it the same through a handle (aceapex_open, whose
    # upload completes before it returns, + aceapex_decode_all_to_host +
    # aceapex_close)
    e2e = None
    if not args.no_e2e:
        h_arc = torch.from_numpy(arc_bytes).pin_memory()
        h_out = torch.empty(N, dtype=torch.uint8).pin_memory()

        def one_call():
            ace.decode_host(h_arc, h_out, device=local)

        def by_handle():
            with ace.Archive(h_arc.numpy(), device=local) as a2:
                a2.decode_all_to_host(h_out, 0, stream)
                stream.synchronize()
                a2.check(stream)

        def e2e_time(fn):
            ts = []
            for i in range(6):
                h_out.zero_()
                torch.cuda.synchronize()
                t = time.perf_counter()
                fn()
                if i >= 3:
                    ts.append(time.perf_counter() - t)
            if not np.array_equal(h_out.numpy(), data):
                raise SystemExit("bench: end-to-end output differs from the input")
            return N / float(np.mean(ts)) / 1e9, len(ts)

        v_handle, _ = e2e_time(by_handle)
        v_one, n_one = e2e_time(one_call)
        e2e = {"value": v_one, "unit": "GB/s", "h2d_bytes_per_step": int(arc_bytes.size),
               "d2h_bytes_per_step": int(N), "steps": n_one,
               "what": "aceapex_decode_host: pinned host archive to pinned host output in one call",
               "open_decode_close_gbs": v_handle}

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_oracle_baseline(arc_bytes, data, "the whole workload")
    if rank == 0:
        config = {"workload": f"paired-end FASTQ {N} bytes, {1 << args.log2_block}-byte blocks, whole-file decode",
                  "log2_block": args.log2_block, "min_match": min_match, "ratio": round(N / arc_bytes.size, 3),
                  "parallelism": f"replicas x{world}", "l2": "inputs larger than L2 (archive and output > 126 MB)",
                  "C_bytes": C, "U_bytes": U, "M_bytes": M, "level_cap": args.max_level, "max_level": st["max_level"],
                  "level_histogram": arc.level_counts(), "encode_seconds": round(enc_s, 2)}
        line = base_line(
            args, value, total_ms / args.steps, world, config,
            roofline={"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                      "peak_kind": peak_kind, "kernel": "decode_kernel", "bytes_model": "C + U + M per launch",
                      "traffic": (recorded_traffic("fastq_1gib_log2B14")
                                  if size == 1 << 30 and args.log2_block == 14 and min_match == 16
                                  and args.max_level == 8 else None),
                      "algorithmic_bytes": C + U + M},
            random_read={"p50_ms": pctl(lat, 50), "p99_ms": pctl(lat, 99), "n": len(lat),
                         "what": "read_lookup + aceapex_decode_range of one FASTQ record, synchronous",
                         "bit_exact": reads_ok, "closure": closure},
            phase_split=phases, batch=batch, serve=serve, level_cap_2=level_cap,
            cpu_baseline=cpu, e2e=e2e, gpu_launches=2 * args.steps, clocks=clk, bit_exact=ok,
            ms_median=float(np.median(step_ms)))
        print(json.dumps(line), flush=True)
    arc.close()
    if world > 1:
        torch.distributed.destroy_process_group()


# -------------------------------------------------------------------- tiny

def workload_tiny(args):
    import torch

    import paper_2606_18900_gb300 as ace
    import synth

    data = synth.tiny_fastq()
    arc_bytes = ace.encode(data, min_match=args.min_match or 16, reads=ace.fastq_index(data))
    arc = ace.Archive(arc_bytes)
    out = torch.empty(data.size, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    run = lambda: arc.decode_all(out, stream)
    for _ in range(args.warmup):
        run()
    arc.check(stream)
    ok = bool(np.array_equal(out.cpu().numpy(), data))
    step_ms = timed_steps(run, stream, args.steps)
    buf = torch.empty(4096, dtype=torch.uint8, device="cuda")
    lat = []
    for r in range(arc.stats()["n_reads"]):
        torch.cuda.synchronize()
        t = time.perf_counter()
        lo, hi = arc.read_lookup(r)
        arc.decode_range(lo, hi, buf, stream)
        stream.synchronize()
        lat.append((time.perf_counter() - t) * 1e3)
    arc.check(stream)
    total_ms = float(sum(step_ms))
    line = base_line(args, data.size * args.steps / (total_ms * 1e-3) / 1e9, total_ms / args.steps, 1,
                     {"workload": f"tiny FASTQ, 2,000 reads, {data.size} bytes (L2-resident: no roofline claim)",
                      "ratio": round(data.size / arc_bytes.size, 3)},
                     random_read={"p50_ms": pctl(lat, 50), "p99_ms": pctl(lat, 99), "n": len(lat)},
                     gpu_launches=2 * args.steps, bit_exact=ok)
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- entropy

# Warp instructions one literal step needs at least (32 symbols): slot mask,
# table address, table load, frequency and bias extraction (4), state shift,
# multiply-add, renormalisation compare, ballot, lane-mask and popc for the
# word index, ring index mask and address, ring load, word insertion (2),
# popc and add for the word pointer, cursor compare and branch, output
# address (2), byte store.
RANS_STEP_OPS = 27


def workload_entropy(args):
    """The entropy stage alone: a literal-only archive (no matches) of
    back-to-back FASTQ quality strings, 16,384 streams of 64 KiB (1 GiB, the
    size of the FASTQ workload) by default, each 16 KiB segment one 32-lane
    interleaved rANS message of 16,384 symbols. (At 256 MiB a launch holds
    only 3.4 segments per warp, and the launch's tail weighs on the rate.)"""
    import torch

    import paper_2606_18900_gb300 as ace
    import synth

    size = args.size or 16384 * 65536
    data = synth.qualities(size)
    t = time.perf_counter()
    arc_bytes = ace.encode(data, log2_B=args.log2_block, min_match=255)
    enc_s = time.perf_counter() - t
    arc = ace.Archive(arc_bytes)
    st = arc.stats()
    if st["match_bytes"] != 0:
        raise SystemExit("bench: the entropy workload must have no matches")
    out = torch.empty(size, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    run = lambda: arc.decode_all(out, stream)
    for _ in range(args.warmup):
        run()
    arc.check(stream)
    ok = bool(np.array_equal(out.cpu().numpy(), data))
    if not ok:
        raise SystemExit("bench: GPU output differs from the input")
    clocks = Clocks(0)
    clocks.start()
    sustain(run, 0.4)
    step_ms = timed_steps(run, stream, args.steps)
    sustain(run, 0.4)
    clk = clocks.stop()
    arc.check(stream)
    total_ms = float(sum(step_ms))
    avg_s = total_ms / args.steps * 1e-3
    sym_s = size / avg_s
    props = torch.cuda.get_device_properties(0)
    mhz = clk["sm_max_mhz"] if clk and clk.get("sm_max_mhz") else 2070.0
    peak_sym = props.multi_processor_count * 4 * mhz * 1e6 / RANS_STEP_OPS * 32
    C, U = st["compressed_bytes"], st["decoded_bytes"]
    peak_hbm, kind = read_peaks()
    config = {"workload": f"entropy stage alone: {size // 65536} x 64 KiB literal-only streams of FASTQ quality "
                          f"symbols ({1 << args.log2_block}-byte segments, no matches)",
              "bits_per_symbol": round(8 * C / U, 3), "C_bytes": C, "U_bytes": U, "encode_seconds": round(enc_s, 2),
              "l2": "inputs larger than L2"}
    line = base_line(args, size * args.steps / (total_ms * 1e-3) / 1e9, total_ms / args.steps, 1, config,
                     symbols_per_s=sym_s,
                     roofline={"bound": "alu", "achieved": sym_s / 1e9, "peak": peak_sym / 1e9, "unit": "Gsymbols/s",
                               "frac": sym_s / peak_sym, "peak_kind": f"issue-limited model: {RANS_STEP_OPS} warp "
                               f"instructions per 32 symbols, {props.multi_processor_count} SMs x 4 schedulers x "
                               f"{mhz:.0f} MHz", "traffic": None, "kernel": "decode_kernel"},
                     hbm_frac=(C + U) / avg_s / 1e9 / peak_hbm, gpu_launches=2 * args.steps, clocks=clk,
                     bit_exact=ok, ms_median=float(np.median(step_ms)))
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ fastq streams

def workload_fastq_streams(args):
    """The paired-end FASTQ stored as four archives of its line streams
    (headers, sequences, '+' lines, qualities): ratio against the single
    archive, and the whole-file decode (a persistent launch per part, device
    newline index, record interleave)."""
    import torch

    import paper_2606_18900_gb300 as ace
    import synth

    size = args.size or (1 << 30)
    data = synth.pe_fastq(size)
    N = data.size
    t = time.perf_counter()
    streams, n_rec = ace.fastq_split(data)
    split_s = time.perf_counter() - t
    t = time.perf_counter()
    arcs = [ace.encode(x, min_match=args.min_match or 16) for x in streams]
    enc_s = time.perf_counter() - t
    single = ace.encode(data, min_match=args.min_match or 16)
    parts = [ace.Archive(a) for a in arcs]
    out = torch.empty(N, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    run = lambda: ace.decode_fastq_streams(parts, out, stream)
    for _ in range(args.warmup):
        run()
    for p_ in parts:
        p_.check(stream)
    ok = bool(np.array_equal(out.cpu().numpy(), data))
    if not ok:
        raise SystemExit("bench: reassembled FASTQ differs from the input")
    step_ms = timed_steps(run, stream, args.steps)
    for p_ in parts:
        p_.check(stream)
    total_ms = float(sum(step_ms))
    comp = sum(int(a.size) for a in arcs)
    line = base_line(args, N * args.steps / (total_ms * 1e-3) / 1e9, total_ms / args.steps, 1,
                     {"workload": f"paired-end FASTQ {N} bytes as four line-stream archives, whole-file decode",
                      "records": n_rec, "stream_bytes": [int(x.size) for x in streams],
                      "archive_bytes": [int(a.size) for a in arcs],
                      "ratio_streams": round(N / comp, 3), "ratio_single_archive": round(N / single.size, 3),
                      "ratio_gain_pct": round(100 * (single.size / comp - 1), 1),
                      "split_seconds": round(split_s, 2), "encode_seconds": round(enc_s, 2),
                      "l2": "inputs larger than L2"},
                     gpu_launches=args.steps * (2 * 4 + 3 * 4 + 1), bit_exact=ok, ms_median=float(np.median(step_ms)))
    print(json.dumps(line), flush=True)
    for p_ in parts:
        p_.close()


# ------------------------------------------------------------------ encode

def workload_encode(args):
    """The GPU encoder on the paired-end FASTQ (1 GiB, 16 KiB blocks,
    min_match 16, read index), or with --encode-input fasta on the FASTA
    genome generator (2 GB, min_match 32: sampled hashing, D = 1 GiB: two
    parse windows). value: input bytes encoded per second with the
    input resident in device memory (device time of each call up to the
    archive's copy-out, CUDA events on the encoder's stream); e2e: host input
    to host archive through the public call. Beside it the library's CPU
    encoder on every host core, whose archive must be identical, and the
    oracle's encoder on a bounded sample."""
    import torch

    import oracle
    import paper_2606_18900_gb300 as ace
    import synth

    fasta = args.encode_input == "fasta"
    size = args.size or (2_000_000_000 if fasta else 1 << 30)
    mm = args.min_match or (32 if fasta else 16)
    data = synth.fasta(size, seed=4) if fasta else synth.pe_fastq(size)
    N = data.size
    reads = None if fasta else ace.fastq_index(data)
    d_in = torch.from_numpy(data).cuda()
    enc = ace.GpuEncoder(0)
    kw = dict(log2_B=args.log2_block, min_match=mm, reads=reads, dist_bound=(1 << 30) if fasta else 0)
    for _ in range(args.warmup):
        arc = enc.encode(d_in, **kw)
    clocks = Clocks(0)
    clocks.start()
    stats = []
    for _ in range(args.steps):
        arc = enc.encode(d_in, **kw)
        stats.append(dict(enc.last_stats))
    clk = clocks.stop()
    dev_ms = [s_["ms_total"] - s_["ms_d2h"] for s_ in stats]
    total_ms = float(sum(dev_ms))
    value = N * args.steps / (total_ms * 1e-3) / 1e9

    e2e = None
    if not args.no_e2e:
        h_in = torch.from_numpy(data).pin_memory().numpy()
        ts = []
        for _ in range(3):
            t = time.perf_counter()
            a2 = enc.encode(h_in, **kw)
            ts.append(time.perf_counter() - t)
        if a2.tobytes() != arc.tobytes():
            raise SystemExit("bench: host-input and device-input encodes differ")
        e2e = {"value": N / float(np.mean(ts)) / 1e9, "unit": "GB/s", "h2d_bytes_per_step": int(N),
               "d2h_bytes_per_step": int(arc.size), "steps": len(ts),
               "what": "GpuEncoder.encode of a pinned host array, archive returned in host memory"}

    t = time.perf_counter()
    host = ace.encode(data, **kw)
    host_s = time.perf_counter() - t
    identical = host.tobytes() == arc.tobytes()
    if not identical:
        raise SystemExit("bench: GPU archive differs from the CPU encoder's")
    with ace.Archive(arc) as a:
        st = a.stats()
        out = torch.empty(N, dtype=torch.uint8, device="cuda")
        a.decode_all(out)
        a.check()
        round_trip = bool(np.array_equal(out.cpu().numpy(), data))
    if not round_trip:
        raise SystemExit("bench: GPU decode of the GPU archive differs from the input")

    cpu = None
    if not args.no_cpu:
        sample = data[: 8 << 20]
        t = time.perf_counter()
        oarc = oracle.encode(sample, log2_B=args.log2_block, min_match=mm, D=kw["dist_bound"])
        o_s = time.perf_counter() - t
        cpu = {"value": sample.size / o_s / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": f"the oracle's encoder on the first {sample.size} bytes of the workload ({o_s:.1f} s)",
               "round_trip": bool(np.array_equal(oracle.decode(oarc), sample)),
               "library_cpu_encoder": {"value": N / host_s / 1e9, "unit": "GB/s",
                                       "cores": len(os.sched_getaffinity(0)), "seconds": round(host_s, 2),
                                       "kind": "aceapex_encode on every host core (same archive)"}}

    match_ms = float(np.mean([s_["ms_match"] for s_ in stats]))  # all windows of one encode
    n_cmd = st["n_commands"]
    # per encode: the sorted (key, position) pairs of every chain window (D
    # bytes of history before each 1 GiB parse window), the input at each
    # position and its 8-byte match-table entry
    D = kw["dist_bound"]
    chunk = max(1 << 30, 1 << min(args.log2_block, 14)) if D else max(N, 1)
    sorted_pairs = sum(min(N, a + chunk) - (max(0, a - D) if D else 0) for a in range(0, N, chunk))
    alg = 8 * sorted_pairs + N + 8 * N
    peak, peak_kind = read_peaks()
    achieved = alg / (match_ms * 1e-3) / 1e9
    mean = lambda k: float(np.mean([s_[k] for s_ in stats]))
    line = base_line(
        args, value, total_ms / args.steps, 1,
        {"workload": (f"GPU encode of FASTA genome {N} bytes, {1 << args.log2_block}-byte blocks, min_match {mm},"
                      f" D = 1 GiB" if fasta else
                      f"GPU encode of paired-end FASTQ {N} bytes, {1 << args.log2_block}-byte blocks, min_match {mm},"
                      " read index"), "log2_block": args.log2_block, "min_match": mm,
         "windows": stats[-1]["windows"],
         "ratio": round(N / arc.size, 3), "archive_bytes": int(arc.size), "n_commands": int(n_cmd),
         "l2": "inputs larger than L2 (input, sort arrays and match table all > 126 MB)",
         "phase_ms": {"hash_and_sort": mean("ms_chains"), "match_kernel": mean("ms_match"),
                      "mask_parse_symbols_levels_deps": mean("ms_parse"),
                      "entropy_and_layout": mean("ms_entropy"), "h2d_copy": mean("ms_h2d"),
                      "archive_d2h": mean("ms_d2h")},
         "identical_to_cpu_encoder": identical, "round_trip": round_trip},
        metric="encoded input GB/s, input resident in device memory",
        roofline={"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                  "peak_kind": peak_kind, "kernel": "enc_match_kernel",
                  "bytes_model": "8 B per sorted (hash, position) pair of every chain window + N input bytes"
                                 " + 8N match table, per encode (all windows' launches)",
                  "algorithmic_bytes": int(alg), "traffic": None,
                  "note": "the input reads at candidate positions are random: latency-bound"},
        cpu_baseline=cpu, e2e=e2e, gpu_launches=int(sum(s_["kernel_launches"] for s_ in stats)), clocks=clk,
        bit_exact=identical and round_trip, ms_median=float(np.median(dev_ms)))
    print(json.dumps(line), flush=True)
    enc.close()


# ------------------------------------------------------------------- batch

def batch_compare(count, max_bytes, steps, min_match=16, tune=True, key=None):
    """`count` independent paired-end FASTQ archives of log-uniform sizes
    16 KiB..max_bytes decoded (a) by one persistent launch replayed from a
    CUDA graph and (b) by one decode call per archive; both bit-exact."""
    import torch

    import paper_2606_18900_gb300 as ace
    from paper_2606_18900_gb300 import autotune
    import synth

    sizes = synth.batch_sizes(count, hi=max_bytes)
    t = time.perf_counter()
    datas = synth.batch_fastq(sizes)
    gen_s = time.perf_counter() - t
    t = time.perf_counter()
    with ThreadPoolExecutor(os.cpu_count() or 1) as ex:
        arcs_b = list(ex.map(lambda d: ace.encode(d, min_match=min_match, threads=1), datas))
    enc_s = time.perf_counter() - t
    total = int(sum(d.size for d in datas))
    handles = [ace.Archive(a) for a in arcs_b]
    offs = np.concatenate([[0], np.cumsum([d.size for d in datas])]).astype(np.int64)
    big = torch.empty(total, dtype=torch.uint8, device="cuda")
    outs = [big[offs[i]:offs[i + 1]] for i in range(len(datas))]
    stream = torch.cuda.Stream()
    batch_run = lambda: ace.decode_batch(handles, outs, stream)
    tuned = None
    if tune:
        tuned, _ = autotune.tune(handles[0], batch_run, key=key or f"batch:{count}:{max_bytes}", stream=stream,
                                 reps=2)
    for _ in range(3):
        batch_run()
    handles[0].check(stream)
    host = big.cpu().numpy()
    ok = all(np.array_equal(host[offs[i]:offs[i + 1]], datas[i]) for i in range(len(datas)))
    # one persistent launch per call, replayed from a CUDA graph
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        batch_run()
    with torch.cuda.stream(stream):
        step_ms = timed_steps(g.replay, stream, steps)
    handles[0].check(stream)
    # one launch per archive
    for h in handles:
        h.set_launch(*(tuned[k] for k in ("ctas", "warps_per_cta", "stage_bytes")) if tuned else ())
    per_run = lambda: [h.decode_all(o, stream) for h, o in zip(handles, outs)]
    per_run()
    stream.synchronize()
    per_ms = timed_steps(per_run, stream, max(1, min(steps, 3)))
    for h in handles:
        h.check(stream)
    host2 = big.cpu().numpy()
    ok &= all(np.array_equal(host2[offs[i]:offs[i + 1]], datas[i]) for i in range(len(datas)))
    for h in handles:
        h.close()
    gb = total / 1e9
    ms = float(np.mean(step_ms))
    return {"archives": len(datas), "total_bytes": total, "max_bytes": max_bytes,
            "one_launch_gbs": gb / (ms * 1e-3), "one_launch_ms": ms, "one_launch_p99_ms": pctl(step_ms, 99),
            "per_archive_gbs": gb / (float(np.mean(per_ms)) * 1e-3), "per_archive_ms": float(np.mean(per_ms)),
            "per_archive_launches": 2 * len(datas), "speedup": float(np.mean(per_ms)) / ms,
            "autotuned_launch": tuned, "generate_seconds": round(gen_s, 1), "encode_seconds": round(enc_s, 1),
            "bit_exact": bool(ok)}


def workload_batch(args):
    r = batch_compare(args.batch_count, args.batch_max, args.steps, args.min_match or 16, not args.no_tune)
    line = base_line(args, r["one_launch_gbs"], r["one_launch_ms"], 1,
                     {"workload": f"{r['archives']} paired-end FASTQ archives, log-uniform 16 KiB-{args.batch_max} B, "
                                  f"{r['total_bytes']} bytes total, one persistent launch from a CUDA graph",
                      "total_bytes": r["total_bytes"], "generate_seconds": r["generate_seconds"],
                      "encode_seconds": r["encode_seconds"], "autotuned_launch": r["autotuned_launch"]},
                     one_launch_per_archive={"gbs": r["per_archive_gbs"], "ms": r["per_archive_ms"],
                                             "launches": r["per_archive_launches"]},
                     speedup_vs_per_archive=r["speedup"], gpu_launches=2 * args.steps, bit_exact=r["bit_exact"])
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ genome

def workload_genome(args):
    import torch

    import paper_2606_18900_gb300 as ace
    import synth

    N = args.size or 50_000_000_000
    t = time.perf_counter()
    data = synth.fasta(N, seed=4)
    gen_s = time.perf_counter() - t
    D = 1 << 30
    t = time.perf_counter()
    cidx, width = ace.fasta_index(data)  # chr:pos coordinate index, stored as the archive's read index
    arc_bytes = ace.encode(data, log2_B=args.log2_block, min_match=args.min_match or 32, dist_bound=D, reads=cidx)
    enc_s = time.perf_counter() - t
    arc = ace.Archive(arc_bytes)
    st = arc.stats()
    stream = torch.cuda.Stream()
    window = args.window
    ring = args.ring
    nw = (N + window - 1) // window
    crc = torch.zeros(nw, dtype=torch.int32, device="cuda")
    run = lambda: arc.stream_range(0, N, ring, window, crc, stream)
    run()
    arc.check(stream)
    got = [int(c) & 0xFFFFFFFF for c in crc.cpu().tolist()]
    with ThreadPoolExecutor(os.cpu_count() or 1) as ex:
        want = list(ex.map(lambda k: zlib.crc32(memoryview(data[k * window:min(N, (k + 1) * window)])), range(nw)))
    ok = got == want
    step_ms = timed_steps(run, stream, args.steps)
    arc.check(stream)
    ms = float(np.mean(step_ms))
    C, U, M = st["compressed_bytes"], st["decoded_bytes"], st["match_bytes"]
    peak, peak_kind = read_peaks()
    achieved = (C + U + M) / (ms * 1e-3) / 1e9
    # regions
    starts = synth.uniform(4, 1, args.regions, N - 150)
    buf = torch.empty(256, dtype=torch.uint8, device="cuda")
    lat = []
    reg_ok = True
    for k, s0 in enumerate(starts):
        s0 = int(s0)
        torch.cuda.synchronize()
        t = time.perf_counter()
        arc.decode_range(s0, s0 + 150, buf, stream)
        stream.synchronize()
        lat.append((time.perf_counter() - t) * 1e3)
        if k < 64:
            reg_ok &= bytes(buf[:150].cpu().numpy()) == data[s0:s0 + 150].tobytes()
    arc.check(stream)
    # the same region lookups by coordinates (record, position) through the
    # coordinate index: bases only, newlines dropped on the device
    n_rec = len(cidx) // 2
    rec_end = [int(cidx[2 * k + 2]) if 2 * k + 2 < len(cidx) else N for k in range(n_rec)]
    bases = [(e - int(cidx[2 * k + 1])) - (e - int(cidx[2 * k + 1]) + width) // (width + 1)
             for k, e in enumerate(rec_end)]
    rng = np.random.default_rng(41)
    coord_lat, coord_ok = [], True
    for k in range(min(args.regions, 10_000)):
        chrom = int(rng.integers(0, n_rec))
        if bases[chrom] < 150:
            continue
        p0 = int(rng.integers(0, bases[chrom] - 150))
        torch.cuda.synchronize()
        t = time.perf_counter()
        arc.decode_region(chrom, p0, 150, buf, width, stream)
        stream.synchronize()
        coord_lat.append((time.perf_counter() - t) * 1e3)
        if k < 64:
            lo, hi = arc.region_lookup(chrom, p0, 150, width)
            coord_ok &= bytes(buf[:150].cpu().numpy()) == data[lo:hi].tobytes().replace(b"\n", b"")
    arc.check(stream)
    # the same byte regions batched: all submitted at once to the serving
    # engine, which decodes the union of their closures per batch
    nb = min(args.regions, 20_000)
    outs = torch.empty((nb, 160), dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    with ace.Server([arc], mem_budget=8 << 30, slots=4) as srv:
        t = time.perf_counter()
        tickets = [srv.submit(0, int(s0), int(s0) + 150, outs[i]) for i, s0 in enumerate(starts[:nb])]
        blat = [srv.wait(tk) for tk in tickets]
        b_s = time.perf_counter() - t
        bst = srv.stats()
    b_ok = all(bytes(outs[i, :150].cpu().numpy()) == data[int(s0):int(s0) + 150].tobytes()
               for i, s0 in enumerate(starts[:64]))
    batched = {"regions_per_s": nb / b_s, "p50_ms": pctl(blat, 50), "p99_ms": pctl(blat, 99), "n": nb,
               "batches": bst["batches"], "bit_exact": bool(b_ok),
               "what": "all regions submitted at once to aceapex_server_submit (latency includes queueing)",
               "serial_regions_per_s": 1e3 / float(np.mean(lat)) if lat else None}
    line = base_line(args, N / (ms * 1e-3) / 1e9, ms, 1,
                     {"workload": f"FASTA genome {N} bytes, D = 1 GiB, streamed through a {ring}-byte device ring "
                                  f"in {window}-byte windows with a CRC-32 per window",
                      "ratio": round(N / arc_bytes.size, 3), "archive_bytes": int(arc_bytes.size),
                      "generate_seconds": round(gen_s, 1), "encode_seconds": round(enc_s, 1),
                      "C_bytes": C, "U_bytes": U, "M_bytes": M},
                     roofline={"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                               "frac": achieved / peak, "peak_kind": peak_kind, "traffic": None,
                               "kernel": "decode_kernel (ring) + CRC kernels", "bytes_model": "C + U + M per stream"},
                     random_read={"p50_ms": pctl(lat, 50), "p99_ms": pctl(lat, 99), "n": len(lat),
                                  "what": "150-byte region, aceapex_decode_range, synchronous", "bit_exact": reg_ok},
                     coordinate_region={"p50_ms": pctl(coord_lat, 50), "p99_ms": pctl(coord_lat, 99),
                                        "n": len(coord_lat), "bit_exact": bool(coord_ok),
                                        "what": "150 bases at (record, position), aceapex_decode_region, synchronous"},
                     batched_regions=batched, crc_windows_match=ok, gpu_launches=args.steps * (1 + 3 * nw),
                     bit_exact=bool(ok and reg_ok and coord_ok and b_ok))
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------- serve

def serve_compare(G, rates, n, budget, slots, serial_n=300, seed=5):
    """Continuous-batching server over the 2,000-read FASTQ and a G-byte
    FASTA genome, both resident: for each offered rate, n requests (90% read
    lookups, 10% ranges log-uniform 1 KiB-64 MiB) arrive with Poisson gaps,
    offered from the library's own submitting thread; against serial
    per-request decode of the same requests (one at a time, synchronous)."""
    import torch

    import paper_2606_18900_gb300 as ace
    import synth

    fq = synth.tiny_fastq()
    t = time.perf_counter()
    fa = synth.fasta(G, seed=seed)
    a_fq = ace.Archive(ace.encode(fq, min_match=16, reads=ace.fastq_index(fq)))
    a_fa = ace.Archive(ace.encode(fa, min_match=32, dist_bound=1 << 30))
    setup_s = time.perf_counter() - t
    src = [fq, fa]
    results = {}
    served, reqs, outs = [], [], []
    for rate in rates:
        rng = np.random.default_rng(int(rate))
        reqs = []
        for _ in range(n):
            if rng.random() < 0.9:
                lo, hi = a_fq.read_lookup(int(rng.integers(0, 2000)))
                reqs.append((0, lo, hi))
            else:
                L = int(np.exp(rng.uniform(np.log(1024), np.log(min(64 << 20, G // 2)))))
                lo = int(rng.integers(0, G - L))
                reqs.append((1, lo, lo + L))
        gaps = synth.poisson_gaps_ns(seed, int(rate), n, rate)
        outs = [torch.empty(hi - lo, dtype=torch.uint8, device="cuda") for _, lo, hi in reqs]
        with ace.Server([a_fq, a_fa], mem_budget=budget, slots=slots) as srv:
            t0 = time.perf_counter()
            tickets, status, t_sub = srv.replay(reqs, outs, gaps)
            lat = [srv.wait(tk) for tk in tickets if tk]
            wall = time.perf_counter() - t0
            st = srv.stats()
        served = [i for i in range(n) if tickets[i]]
        total_bytes = sum(reqs[i][2] - reqs[i][1] for i in served)
        torch.cuda.synchronize()
        ok = all(np.array_equal(outs[i].cpu().numpy(), src[reqs[i][0]][reqs[i][1]:reqs[i][2]])
                 for i in served[:: max(1, len(served) // 200)])
        results[str(int(rate))] = {"p50_ms": pctl(lat, 50), "p99_ms": pctl(lat, 99), "gbs": total_bytes / wall / 1e9,
                                   "offered_rate": rate, "achieved_submit_rate": n / t_sub if t_sub else None,
                                   "served": len(served), "batches": st["batches"], "max_batch": st["max_batch"],
                                   "max_inflight": st["max_inflight"], "refused": st["refused"],
                                   "bytes": total_bytes, "bit_exact_sample": ok}
    # serial per-request decode (one request at a time, synchronous)
    stream = torch.cuda.Stream()
    arcs = [a_fq, a_fa]
    lat_s, nbytes = [], 0
    t0 = time.perf_counter()
    for (a, lo, hi), o in [(reqs[i], outs[i]) for i in served][:serial_n]:
        t = time.perf_counter()
        arcs[a].decode_range(lo, hi, o, stream)
        stream.synchronize()
        lat_s.append((time.perf_counter() - t) * 1e3)
        nbytes += hi - lo
    serial_s = time.perf_counter() - t0
    for a in arcs:
        a.check(stream)
        a.close()
    return {"genome_bytes": G, "budget_bytes": budget, "slots": slots, "setup_seconds": round(setup_s, 1),
            "rates": results, "serial_per_request": {"p50_ms": pctl(lat_s, 50), "p99_ms": pctl(lat_s, 99),
                                                     "gbs": nbytes / serial_s / 1e9, "n": len(lat_s)}}


def workload_serve(args):
    G = args.size or 3_000_000_000
    r = serve_compare(G, [float(x) for x in args.rates.split(",")], args.requests, args.budget, args.slots)
    best = max(r["rates"].values(), key=lambda v: v["gbs"])
    line = base_line(args, best["gbs"], None, 1,
                     {"workload": f"serving: tiny FASTQ + {G}-byte genome resident; Poisson arrivals, 90% read "
                                  "lookups / 10% ranges log-uniform 1 KiB-64 MiB, offered from the library's "
                                  "submitting thread",
                      "budget_bytes": args.budget, "slots": args.slots, "setup_seconds": r["setup_seconds"]},
                     rates=r["rates"], serial_per_request=r["serial_per_request"],
                     gpu_launches=None, bit_exact=all(v["bit_exact_sample"] for v in r["rates"].values()))
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------- reference

def run_reference(args):
    """The CPU oracle, as it stands, timed on the host cores on a bounded
    sample of the workload (the paper's comparison systems are out of scope)."""
    if int(os.environ.get("RANK", "0")) != 0:
        return
    import oracle
    import paper_2606_18900_gb300 as ace
    import synth

    if args.workload == "encode":
        run_reference_encode(args)
        return
    sample = min(args.size or (1 << 30), 96 << 20)
    if args.workload == "genome":
        data = synth.fasta(sample, seed=4)
        args.min_match = args.min_match or 32
    elif args.workload == "tiny":
        data = synth.tiny_fastq()
    else:
        data = synth.pe_fastq(args.size or (1 << 30))[:sample].copy()
    arc = ace.encode(data, log2_B=args.log2_block, min_match=args.min_match or 16)
    for _ in range(args.warmup):
        oracle.decode(arc)
    ts = []
    for _ in range(args.steps):
        t = time.perf_counter()
        out = oracle.decode(arc)
        ts.append(time.perf_counter() - t)
    assert np.array_equal(out, data)
    total = sum(ts)
    v = data.size * args.steps / total / 1e9
    cores = len(os.sched_getaffinity(0))
    size = args.size or (1 << 30)
    names = {"fastq": f"paired-end FASTQ {size} bytes, {1 << args.log2_block}-byte blocks, whole-file decode",
             "genome": f"FASTA genome {args.size or 50_000_000_000} bytes, D = 1 GiB, streamed through a device ring",
             "tiny": "tiny FASTQ, 2,000 reads"}
    line = base_line(args, v, 1e3 * total / args.steps, args.gpus,
                     {"workload": names.get(args.workload, args.workload), "log2_block": args.log2_block,
                      "sample": f"each step decodes the first {data.size} bytes of the workload"},
                     impl="reference",
                     cpu_baseline={"value": v, "unit": "GB/s", "cores": 1, "kind": "oracle",
                                   "sample": f"first {data.size} bytes of the workload per step; host has {cores} cores"},
                     e2e={"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0})
    print(json.dumps(line), flush=True)


def run_reference_encode(args):
    """The oracle's encoder, as it stands, on the first 8 MiB of the encode
    workload per step (its speed makes the whole 1 GiB take minutes)."""
    import oracle
    import synth

    size = args.size or (1 << 30)
    mm = args.min_match or 16
    data = synth.pe_fastq(size)[: min(size, 8 << 20)].copy()
    for _ in range(args.warmup):
        oracle.encode(data, log2_B=args.log2_block, min_match=mm)
    ts = []
    for _ in range(args.steps):
        t = time.perf_counter()
        arc = oracle.encode(data, log2_B=args.log2_block, min_match=mm)
        ts.append(time.perf_counter() - t)
    assert np.array_equal(oracle.decode(arc), data)
    total = sum(ts)
    v = data.size * args.steps / total / 1e9
    cores = len(os.sched_getaffinity(0))
    line = base_line(args, v, 1e3 * total / args.steps, args.gpus,
                     {"workload": f"GPU encode of paired-end FASTQ {size} bytes, {1 << args.log2_block}-byte blocks,"
                                  f" min_match {mm}, read index", "log2_block": args.log2_block, "min_match": mm,
                      "sample": f"each step encodes the first {data.size} bytes of the workload"},
                     metric="encoded input GB/s, input resident in device memory", impl="reference",
                     cpu_baseline={"value": v, "unit": "GB/s", "cores": 1, "kind": "oracle",
                                   "sample": f"first {data.size} bytes of the workload per step; host has {cores} cores"},
                     e2e={"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0})
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.phase_child:
        phase_child(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload == "fastq":
        workload_fastq(args)
    elif args.workload == "tiny":
        workload_tiny(args)
    elif args.workload == "batch":
        workload_batch(args)
    elif args.workload == "serve":
        workload_serve(args)
    elif args.workload == "entropy":
        workload_entropy(args)
    elif args.workload == "fastq_streams":
        workload_fastq_streams(args)
    elif args.workload == "encode":
        workload_encode(args)
    else:
        workload_genome(args)


if __name__ == "__main__":
    main()
