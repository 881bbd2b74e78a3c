"""Benchmark: device-resident whole-file decode of the 1 GiB paired-end FASTQ
workload (16 KiB blocks), decompressed GB/s, with the HBM roofline fraction
of the decode kernel, an end-to-end figure through the C ABI with host
buffers, and the CPU oracle decoder timed on this host's cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--log2-block 14|20] [--size BYTES]

One JSON line on rank 0. Multi-GPU runs (torchrun) decode one replica of the
workload per GPU (whole-file decode does not shard: replicas only) and report
the aggregate over ranks.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--log2-block", type=int, default=14)
    p.add_argument("--size", type=int, default=1 << 30)
    p.add_argument("--min-match", type=int, default=16)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    return p.parse_args()


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampler running during the timed region."""

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
        sm, mx, reasons = [], 0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx = max(mx, float(f[2]))
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
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def make_workload(size, log2_block, min_match, rank, world):
    """1 GiB paired-end FASTQ (seed 2) encoded by the library encoder. With
    several ranks, rank 0 encodes once and shares the archive via /dev/shm."""
    import paper_2606_18900_gb300 as ace
    import synth

    data = synth.pe_fastq(size)
    path = f"/dev/shm/aceapex_bench_{size}_{log2_block}_{min_match}.bin"
    if world > 1 and rank != 0:
        import torch.distributed as dist
        dist.barrier()
        arc = np.fromfile(path, dtype=np.uint8)
        return data, arc
    t = time.perf_counter()
    arc = ace.encode(data, log2_B=log2_block, min_match=min_match, reads=ace.fastq_index(data))
    enc_s = time.perf_counter() - t
    if world > 1:
        import torch.distributed as dist
        arc.tofile(path)
        dist.barrier()
    make_workload.encode_seconds = enc_s
    return data, arc


def cpu_oracle_baseline(arc, data, budget_s=25.0):
    """The CPU oracle decoder as it stands, single-threaded, on the whole
    archive (one pass is ~10-30 s of CPU work at this size)."""
    import oracle

    t = time.perf_counter()
    out = oracle.decode(arc)
    dt = time.perf_counter() - t
    ok = bool(np.array_equal(out, data))
    return {"value": data.size / dt / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": f"whole archive, one sequential pass ({data.size} bytes, {dt:.1f} s)", "bit_exact": ok}


def run_reference(args):
    """The CPU oracle timed as the reference arm on bounded samples."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    import paper_2606_18900_gb300 as ace
    import synth

    sample = min(args.size, 96 << 20)
    data = synth.pe_fastq(args.size)[:sample].copy()
    arc = ace.encode(data, log2_B=args.log2_block, min_match=args.min_match)
    for _ in range(args.warmup):
        oracle.decode(arc)
    ts = []
    for _ in range(args.steps):
        t = time.perf_counter()
        out = oracle.decode(arc)
        ts.append(time.perf_counter() - t)
    assert np.array_equal(out, data)
    total = sum(ts)
    v = sample * args.steps / total / 1e9
    cores = len(os.sched_getaffinity(0))
    line = {
        "impl": "reference", "metric": "decompressed GB/s device-resident", "value": v, "unit": "GB/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": f"paired-end FASTQ, first {sample} bytes of the {args.size}-byte workload per step",
                   "log2_block": args.log2_block},
        "cpu_baseline": {"value": v, "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": f"first {sample} bytes of the workload per step; host has {cores} cores"},
        "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch

    import paper_2606_18900_gb300 as ace

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    data, arc_bytes = make_workload(args.size, args.log2_block, args.min_match, rank, world)
    N = data.size
    arc = ace.Archive(arc_bytes, device=local)
    st = arc.stats()
    C, U, M = st["compressed_bytes"], st["decoded_bytes"], st["match_bytes"]
    out = torch.empty(N, dtype=torch.uint8, device=f"cuda:{local}")
    stream = torch.cuda.Stream()

    for _ in range(args.warmup):
        arc.decode_all(out, stream)
    arc.check(stream)
    ok = bool(np.array_equal(out.cpu().numpy(), data))
    if not ok:
        raise SystemExit("bench: GPU output differs from the input")

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = Clocks(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t0 = time.perf_counter()
    for i in range(args.steps):
        ev[i][0].record(stream)
        arc.decode_all(out, stream)
        ev[i][1].record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    arc.check(stream)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = float(sum(step_ms))
    if world > 1:
        t = torch.tensor([total_ms], device=f"cuda:{local}")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    value = N * world * args.steps / (total_ms * 1e-3) / 1e9
    avg_ms = float(np.mean(step_ms))
    peak, peak_kind = read_peaks()
    achieved = (C + U + M) / (avg_ms * 1e-3) / 1e9

    # end to end through the C ABI with host buffers: open (H2D of the archive
    # from pinned memory) + decode + D2H of the output, every step
    e2e = None
    if not args.no_e2e:
        h_arc = torch.from_numpy(arc_bytes).pin_memory()
        h_out = torch.empty(N, dtype=torch.uint8).pin_memory()
        ts = []
        for i in range(6):
            torch.cuda.synchronize()
            t = time.perf_counter()
            with ace.Archive(h_arc.numpy(), device=local) as a2:
                a2.decode_all(out, stream)
                stream.synchronize()
                h_out.copy_(out)
                a2.check(stream)
            if i >= 3:
                ts.append(time.perf_counter() - t)
        e2e = {"value": N / float(np.mean(ts)) / 1e9, "unit": "GB/s", "h2d_bytes_per_step": int(arc_bytes.size),
               "d2h_bytes_per_step": int(N), "steps": len(ts)}

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_oracle_baseline(arc_bytes, data)
        cpu["cores"] = 1
    if rank == 0:
        line = {
            "metric": "decompressed GB/s device-resident", "value": value, "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic",
            "config": {"workload": f"paired-end FASTQ {N} bytes (1 GiB generator), {1 << args.log2_block}-byte blocks, "
                                   "whole-file decode", "log2_block": args.log2_block, "min_match": args.min_match,
                       "ratio": round(N / arc_bytes.size, 3), "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (archive and output > 126 MB)",
                       "C_bytes": C, "U_bytes": U, "M_bytes": M, "max_level": st["max_level"],
                       "encode_seconds": round(getattr(make_workload, "encode_seconds", 0.0), 2)},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_kind": peak_kind, "traffic": None,
                         "kernel": "decode_kernel (begin_kernel negligible)",
                         "bytes_model": "C + U + M per launch"},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": 2 * args.steps,
            "clocks": clk,
            "bit_exact": ok,
            "wall_s_timed": wall,
        }
        print(json.dumps(line), flush=True)
    arc.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
