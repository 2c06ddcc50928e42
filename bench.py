#!/usr/bin/env python3
"""Benchmark of the GB300 BWT build + merge path (and MEM search on its result).

Workload (default): the pangenome merge -- a 5 Mb uniform-random founder, 50
haplotypes with 0.1% SNPs and 0.01% indels, both strands (~500 M symbols),
built incrementally in batches of 10 haplotypes: batch 0 is built, batches 1-4
are each built on the device and merged into the index of the batches before
them (100, 200, 300, 400 Msym).  Timed step k is merge step k mod 4 of such a
pass; every pass starts from its own batch-0 index, built before the timed
region, so every timed step is a step of the workload whatever K.  The steps of
a pass run through rb3_append_batches, which builds batch k+1 while batch k
merges.  value = new symbols per second (Msym/s) over the K timed steps, inputs
resident in HBM.  The finished index (all 50 haplotypes) is then searched for
SMEMs (>= 31 bp) of 1 M queries (lognormal lengths, median 150 bp; 90% from the
haplotypes with 1% substitutions, 10% random) -- reported as `mem_search`
(Mbp/s) beside the plain one-query-per-thread form -- and a batch already in
the index is merged again (`merge_of_indexed_batch`).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl rb3|reference]

With torchrun (N > 1) every rank runs its own independent pangenome (weak
scaling, no data-path collective); rank 0 prints one JSON line.
`--impl reference` times the CPU oracle (plain Algorithm 1 on naive-sort batch
BWTs) on a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOAD = ("pangenome merge: 5 Mb uniform founder, 50 haplotypes (0.1% SNPs, 0.01% indels 1-10 bp), "
            "both strands (~500 Msym), batches of 10 haplotypes; step = device batch-BWT build + merge into "
            "the running index")
METRIC = "BWT-merge Msymbols/s"


# DRAM traffic per launch of the kernel the roofline reports, from one ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum, one pass) of the four
# merges of one pass of the default workload, averaged:
#   ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum --clock-control none
#       -k regex:k_walk_seeded -s 3 -c 4 python bench.py --steps 4 --warmup 3 --no-serve --no-cpu --no-search
#       --no-plain --uneven-genomes 0 --seg-len 1284 --seed-cap 1284
# (the knobs the autotuner picks for this workload; k.merge_walk is k_walk_seeded's phase)
# Keyed by (kernel, Occ interval, founder bp, merge form, segment length, seed
# cap, digest of the merge kernel's sources): a change to the kernel's source
# or other knobs drops the figure (null)
# until it is captured again.  Every timed step is a step of one pass, so the
# per-launch average does not depend on the number of steps (a multiple of 4).
NCU_TRAFFIC: dict = {("k.merge_walk", 32, 5_000_000, 0, 1284, 1284, "f2f4d433d991a70d"): 5.99e9}


def kernel_digest() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in ("merge.cu", "common.cuh"):
        with open(os.path.join(ROOT, "paper_2409_00613_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=4)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["rb3", "reference"], default="rb3")
    p.add_argument("--scale", type=float, default=1.0, help="founder length / 5 Mb (1.0 = the workload)")
    p.add_argument("--queries", type=int, default=1_000_000)
    p.add_argument("--no-search", action="store_true")
    p.add_argument("--no-plain", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--seg-len", type=int, default=0)
    p.add_argument("--seed-cap", type=int, default=0, help="merge: ForwardExt steps of a segment seed (0 = default)")
    p.add_argument("--merge-form", type=int, default=0,
                   help="0: bounded seeds, segment tops at content anchors (default); 2: bounded seeds, tops every "
                        "L symbols; 3: uncapped seeds with the takeover chain, anchored tops")
    p.add_argument("--walk-ctas", type=int, default=0, help="merge walk CTAs per SM (0 = library default)")
    p.add_argument("--occ", type=int, default=32)
    p.add_argument("--no-serve", action="store_true")
    p.add_argument("--uneven-genomes", type=int, default=256,
                   help="uneven-genome leg: the first N genomes (batches of 64) of the 2,000-genome workload, "
                        "layout autotuned (0 = skip)")
    p.add_argument("--serve-full", action="store_true",
                   help="also build the served index (20 haplotypes of a 150 Mb founder, ~6 Gsym) and serve on it")
    return p.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_hint: str | None):
        self.bus = (bus_hint or "").lower()
        self.proc = None
        self.path = os.path.join("/tmp", f"rb3_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                if self.bus and self.bus not in parts[0].lower():
                    continue
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max((num(r[3]) or 0.0) for r in rows)}


def bus_id(torch, dev):
    try:
        p = torch.cuda.get_device_properties(dev)
        return f"{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0"
    except Exception:
        return None


# ---------------------------------------------------------------------------
# the rb3 arm
# ---------------------------------------------------------------------------
def aggregate_ranks(ms, new_syms, world, device):
    """Whole-job figures over the ranks: the slowest rank's time (max) and the
    symbols of all ranks (sum); each rank runs its own replica (weak scaling)."""
    if world == 1:
        return ms, float(new_syms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    s = torch.tensor([float(new_syms)], device=device, dtype=torch.float64)
    dist.all_reduce(s)
    return float(t.item()), float(s.item())


def run_rb3(args, rank, world, local_rank):
    import torch
    import paper_2409_00613_gb300 as rb

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    st = torch.cuda.current_stream()
    founder = int(5_000_000 * args.scale)
    S = synth.pangenome(seed=synth.SEED_BASE + 1 + 1000 * rank, founder_len=founder, n_hap=50, batch=10)
    off = S.offsets
    batches = S.batches
    dev_batches = []
    for (a, b) in batches:
        seq = S.seq[off[a]:off[b]]
        dev_batches.append((torch.from_numpy(seq.copy()).to(dev), S.lens[a:b].copy()))
    ds = [int(2 * (lens.sum() + len(lens))) for (_, lens) in dev_batches]
    opts = {"occ_interval": args.occ, "seg_len": args.seg_len, "walk_ctas_per_sm": args.walk_ctas,
            "merge_form": args.merge_form, "seed_cap": args.seed_cap}
    # The workload is one pass: batch 0 built, batches 1..4 built and merged into
    # an index of 100, 200, 300, 400 Msym.  Timed step k is merge step k mod 4 of
    # a pass; every pass starts from its own batch-0 index, built before the
    # timed region, so that every timed step is a step of the workload whatever K.
    n_merge = len(batches) - 1
    step_batch = [1 + (k % n_merge) for k in range(max(args.steps, args.warmup))]
    groups = [list(range(g0, min(g0 + n_merge, args.steps))) for g0 in range(0, args.steps, n_merge)]

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # batches 1..4 back to back (device, and pinned host for e2e); pass g reads
    # the prefix holding its steps' batches
    s1 = off[batches[1][0]]
    all_seq = S.seq[s1:off[batches[-1][1]]]
    merge_dev = torch.from_numpy(all_seq.copy()).to(dev)
    merge_host = torch.empty(len(all_seq), dtype=torch.uint8, pin_memory=True)
    merge_host.numpy()[:] = all_seq

    def group_args(g):
        bs = [step_batch[k] for k in g]  # 1, 2, ... in order
        a, b = batches[bs[0]][0], batches[bs[-1]][1]
        nbytes = int(off[b] - off[a])
        lens = S.lens[a:b].astype(np.int64)
        ends = np.cumsum([batches[x][1] - batches[x][0] for x in bs]).astype(np.int64)
        return nbytes, lens, ends

    new_syms = int(sum(ds[b] for b in step_batch))

    def fresh_base():
        x = rb.rb3_build_batch(dev_batches[0][0], dev_batches[0][1], opts=opts, stream=st)
        rb.rb3_drop_build_data(x)
        return x

    # ---- device memory of one batch build (peak of the library's allocations, untimed) ----
    torch.cuda.synchronize()
    base_mem = rb.rb3_device_peak(reset=True)
    probe = rb.rb3_build_batch(dev_batches[1][0], dev_batches[1][1], opts=opts, stream=st)
    torch.cuda.synchronize()
    peak_mem = rb.rb3_device_peak()
    probe_bytes = rb.rb3_index_bytes(probe)["device_bytes"]
    probe.free()
    memory = {"batch_symbols": ds[1], "build_peak_bytes_per_symbol": round((peak_mem - base_mem) / ds[1], 1),
              "index_bytes_per_symbol": round(probe_bytes / ds[1], 3),
              "what": "peak of the library's device allocations during one batch build, above what was in use "
                      "before it, per indexed symbol; the batch's index itself (D = 32)"}
    # ---- autotune the merge's segment length on batch 1 into batch 0 (untimed) ----
    tune = {}
    if not args.seg_len:
        idx = fresh_base()
        src = rb.rb3_build_batch(*dev_batches[1], opts=opts, stream=st)
        best, tms = rb.rb3_tune_merge(idx, src, opts, stream=st)
        src.free()
        idx.free()
        opts["seg_len"] = int(best.seg_len)
        opts["seed_cap"] = int(best.seed_cap)
        tune = {"seg_len": int(best.seg_len), "seed_cap": int(best.seed_cap), "walk_ms": round(tms, 3),
                "candidates": "L in {L0/2, L0, 2 L0, 4 L0} (L0 = n2/(SMs*512)) x seed cap in {L, 2L, 4L}"}

    def run_groups(bases, src, host):
        for g, x in zip(groups, bases):
            nbytes, lens, ends = group_args(g)
            rb.rb3_append_batches(x, src[:nbytes], lens, ends, opts, stream=st)

    # ---- warm-up: W steps of the same schedule, untimed ----
    if args.warmup:
        wgroups = [list(range(g0, min(g0 + n_merge, args.warmup))) for g0 in range(0, args.warmup, n_merge)]
        for g in wgroups:
            x = fresh_base()
            nbytes, lens, ends = group_args(g)
            rb.rb3_append_batches(x, merge_dev[:nbytes], lens, ends, opts, stream=st)
            x.free()
    # ---- timed: ceil(K/4) passes, each into its own batch-0 index (built untimed) ----
    bases = [fresh_base() for _ in groups]
    barrier()
    rb.rb3_profile_reset()
    rb.rb3_profile_enable(True)
    rb.rb3_walk_stats(reset=True)
    clocks = ClockSampler(bus_id(torch, local_rank))
    clocks.start()
    launches0 = rb.rb3_launch_count()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    barrier()
    t0.record(st)
    run_groups(bases, merge_dev, False)
    t1.record(st)
    barrier()
    ms = t0.elapsed_time(t1)
    launches = rb.rb3_launch_count() - launches0
    clk = clocks.stop()
    rb.rb3_profile_enable(False)
    prof = rb.rb3_profile_read()
    walk_launch_ms = [round(d, 3) for (nm, _, d) in rb.rb3_profile_timeline() if nm == "k.merge_walk"]
    wstats = rb.rb3_walk_stats()
    # the index the searches use: the last pass, completed (untimed) if K is not a multiple of 4
    idx = bases[-1]
    done = len(groups[-1])
    if done < n_merge:
        rest = [b for b in range(1 + done, len(batches))]
        a, b = batches[rest[0]][0], batches[rest[-1]][1]
        rb.rb3_append_batches(idx, torch.from_numpy(S.seq[off[a]:off[b]].copy()).to(dev),
                              S.lens[a:b].astype(np.int64),
                              np.cumsum([batches[x][1] - batches[x][0] for x in rest]).astype(np.int64), opts,
                              stream=st)
    for x in bases[:-1]:
        x.free()
    info = rb.rb3_index_info(idx)
    ms, total_syms = aggregate_ranks(ms, new_syms, world, dev)
    value = total_syms / (ms * 1e3)

    # ---- one pass one step at a time (build, then merge): no overlap ----
    seq_idx = fresh_base()
    barrier()
    a_ev = torch.cuda.Event(enable_timing=True)
    b_ev = torch.cuda.Event(enable_timing=True)
    a_ev.record(st)
    for b in range(1, len(batches)):
        src = rb.rb3_build_batch(dev_batches[b][0], dev_batches[b][1], opts=opts, stream=st)
        rb.rb3_merge_opts(seq_idx, src, opts, stream=st)
        src.free()
    b_ev.record(st)
    barrier()
    seq_ms = a_ev.elapsed_time(b_ev)
    same = bool(np.array_equal(rb.rb3_export(seq_idx), rb.rb3_export(idx)))
    seq_idx.free()

    # ---- e2e: the public call on pinned host buffers (h2d inside the call) ----
    e2e_bases = [fresh_base() for _ in groups]
    barrier()
    e0 = time.perf_counter()
    run_groups(e2e_bases, merge_host, True)  # each call reads the merged counts back
    torch.cuda.synchronize()
    e_ms = (time.perf_counter() - e0) * 1e3
    for x in e2e_bases:
        x.free()
    h2d = sum(group_args(g)[0] + 8 * len(group_args(g)[1]) for g in groups)
    e2e = {"value": round(new_syms / (e_ms * 1e3), 3), "unit": "Msym/s",
           "h2d_bytes_per_step": int(h2d // max(1, args.steps)), "d2h_bytes_per_step": 96}

    # ---- roofline of the dominant kernel (live CUDA events of the timed region) ----
    hbm, peak_kind = peaks()
    kern = {k: v for k, v in prof.items() if k.startswith("k.") and v[2] > 0}
    roof = None
    if kern:
        # the merge walk: the largest event total of the timed region (the build's kernels
        # run beside it on another stream, so their totals overlap its time)
        top = "k.merge_walk" if "k.merge_walk" in kern else max(kern, key=lambda k: kern[k][0])
        kms, kcalls, kbytes = kern[top]
        achieved = kbytes / (kms * 1e-3) / 1e9
        roof = {"kernel": top, "bound": "hbm", "achieved": round(achieved, 1), "peak": hbm,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / hbm, 4),
                "traffic": (NCU_TRAFFIC.get((top, info["occ_interval"], founder, args.merge_form, opts["seg_len"],
                                             opts["seed_cap"], kernel_digest()))
                            if args.steps % n_merge == 0 else None),
                "kernel_digest": kernel_digest(),
                "algo_bytes_per_launch": kbytes / max(1, kcalls), "avg_launch_ms": kms / max(1, kcalls),
                "launches": kcalls, "share_of_step": round(kms / ms, 4)}
        if top == "k.merge_walk" and info["occ_interval"] == 32:
            # the walk against the random-request roofline: every lane's rank read is
            # one 32-byte access at D = 32, every walk step also writes pos; the
            # ceiling is the probe's dependent-chain random reads on this GPU.
            # Lanes on homologous suffixes that read one sector in one instruction
            # make one memory request, so the lane-level rate can pass the probe's
            req = wstats["seed_block_reads"] + 2 * wstats["walk_block_reads"]
            _, probe_m = rb.rb3_probe_random_gather(32, 1, 2048, 8 << 30, stream=st)
            per_s = req / (kms * 1e-3)
            roof["random_requests"] = {
                "per_launch": req / max(1, kcalls), "G_per_s": round(per_s / 1e9, 2),
                "probe_G_per_s": round(probe_m / 1e3, 2), "frac": round(per_s / (probe_m * 1e6), 3),
                "seeds": wstats["seeds"], "seed_block_reads": wstats["seed_block_reads"],
                "walk_block_reads": wstats["walk_block_reads"], "walked_again": wstats["walked_again"],
                "what": "lane-level rank block reads of the seeds and walk steps plus the walk's pos writes, "
                        "counted by the kernel, over its CUDA-event time; ceiling: rb3_probe_random_gather, "
                        "32-byte dependent random reads, 2048 threads per SM, 8 GiB buffer"}
    phases = {k: round(v[0], 3) for k, v in sorted(prof.items())}

    out = {"metric": METRIC, "value": round(value, 3), "unit": "Msym/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "founder_bp": founder, "haplotypes": 50, "batch_haplotypes": 10,
                      "new_symbols_per_gpu": new_syms, "final_index_symbols": info["n"],
                      "index_symbols_before_step": [int(sum(ds[:b])) for b in step_batch[:n_merge]],
                      "passes": len(groups),
                      "schedule": "timed step k builds batch 1 + (k mod 4) and merges it into the index of "
                                  "batches 0..(k mod 4); every 4 steps a fresh batch-0 index (built untimed)",
                      "occ_interval": info["occ_interval"], "seg_len": opts["seg_len"],
                      "l2": "inputs larger than L2 (batch ~100 Msym text + 100-500 MB index per step)",
                      "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
           "e2e": e2e, "gpu_launches": int(launches), "clocks": clk, "roofline": roof, "phases_ms": phases,
           "walk_ms_per_step": walk_launch_ms,
           "autotune": tune, "memory": memory,
           "one_by_one": {"ms_per_step": round(seq_ms / n_merge, 3),
                          "value": round(sum(ds[1:]) / (seq_ms * 1e3), 3), "unit": "Msym/s",
                          "equal_output": same,
                          "note": "one pass, each step's build then its merge, no overlap (the timed value "
                                  "overlaps the next batch's build with the current merge)"}}

    # ---- a batch whose haplotypes are already in the index ----
    if rank == 0:
        out["merge_of_indexed_batch"] = indexed_batch_merge(rb, torch, dev_batches, opts, st, ds)

    # ---- comparison with the plain one-walk-per-string form on one merge ----
    if not args.no_plain and rank == 0:
        out["merge_vs_plain"] = plain_vs_segmented(rb, torch, dev_batches, opts, st, ds)

    # ---- MEM search on the finished index ----
    if not args.no_search and rank == 0:
        probe = (roof or {}).get("random_requests", {}).get("probe_G_per_s")
        out["mem_search"] = mem_search(rb, torch, S, idx, args, st, dev, probe)
        if not args.no_serve:
            out["mem_search"]["served"] = served(rb, S, idx, "pangenome-merge index (500 Msym)")
        out["run_length"] = run_length_bench(rb, torch, S, idx, args, st, dev,
                                             out["mem_search"]["autotune_chunk_len"])
        out["run_length"]["merge_into"] = rle_merge_bench(rb, torch, dev_batches, opts, st, ds)
        out["haplotype_diversity"] = diversity_bench(rb, torch, S, idx, st, dev, probe)
        out["bwasw"] = bwasw_bench(rb, torch, S, idx, st, dev)
    idx.free()
    if not args.no_search and rank == 0:
        out["locate"] = locate_bench(rb, torch, S, args, st, dev, opts, batches, off)
    if args.serve_full and rank == 0:
        out["served_full"] = served_full(rb, torch, st, dev, opts)
    if args.uneven_genomes and rank == 0:
        out["uneven"] = uneven_bench(rb, torch, st, dev, args.uneven_genomes)
    if rank == 0 and not args.no_cpu and world == 1:
        out["cpu_baseline"] = cpu_sample(S)
        if "haplotype_diversity" in out:
            try:  # a side leg: a failure is recorded, the bench line still printed
                out["haplotype_diversity"]["cpu_baseline"] = diversity_cpu_sample(S)
            except (RuntimeError, OSError, ValueError) as e:
                out["haplotype_diversity"]["cpu_baseline"] = {"error": f"{type(e).__name__}: {e}"}
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


def indexed_batch_merge(rb, torch, dev_batches, opts, st, ds):
    """The merge of a batch whose haplotypes the index already holds (batch 1
    into the index of batches 0-1: every new string equals an indexed one to
    its sentinel), beside the merge of a fresh batch (batch 2) into the same
    index; both outputs checked equal to the index built the other way round."""
    res = {"what": "batch 1 (10 haplotypes already indexed) merged into the index of batches 0-1, against batch 2 "
                   "(fresh haplotypes) into the same index; walk = k.merge_walk's CUDA-event time",
           "new_symbols": ds[1]}
    for name, b in (("indexed", 1), ("fresh", 2)):
        base = rb.rb3_build_batch(*dev_batches[0], opts=opts, stream=st)
        rb.rb3_drop_build_data(base)
        one = rb.rb3_build_batch(*dev_batches[1], opts=opts, stream=st)
        rb.rb3_merge_opts(base, one, opts, stream=st)
        one.free()
        src = rb.rb3_build_batch(*dev_batches[b], opts=opts, stream=st)
        torch.cuda.synchronize()
        rb.rb3_profile_reset()
        rb.rb3_profile_enable(True)
        a = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        a.record(st)
        rb.rb3_merge_opts(base, src, opts, stream=st)
        e.record(st)
        torch.cuda.synchronize()
        rb.rb3_profile_enable(False)
        prof = rb.rb3_profile_read()
        res[f"{name}_merge_ms"] = round(a.elapsed_time(e), 3)
        res[f"{name}_walk_ms"] = round(prof.get("k.merge_walk", (float("nan"),))[0], 3)
        src.free()
        base.free()
    res["indexed_over_fresh_walk"] = round(res["indexed_walk_ms"] / res["fresh_walk_ms"], 2)
    return res


def rle_merge_bench(rb, torch, dev_batches, opts, st, ds, span=2048):
    """The last batch (100 Msym) merged into the index of the batches before it
    (400 Msym), held plain (D = 32) and run-length encoded (span 2048, merged
    into directly): each merge's time (CUDA events around the call) and the
    peak of the library's device allocations during it above what was in use
    before; the two merged BWTs compared on the device."""
    last = len(dev_batches) - 1
    P = rb.rb3_build_batch(*dev_batches[0], opts=opts, stream=st)
    rb.rb3_drop_build_data(P)
    for b in range(1, last):
        src = rb.rb3_build_batch(*dev_batches[b], opts=opts, stream=st)
        rb.rb3_merge_opts(P, src, opts, stream=st)
        src.free()
    R = rb.rb3_index_compress(P, span, stream=st)
    res = {"what": f"batch {last} ({ds[last]} symbols) merged into the index of batches 0-{last - 1} "
                   f"({sum(ds[:last])} symbols), plain D = 32 and run-length span {span}; peak = the library's "
                   "device allocations during the call above those before it", "span": span}
    for name, dst in (("plain", P), ("run_length", R)):
        src = rb.rb3_build_batch(*dev_batches[last], opts=opts, stream=st)
        before = rb.rb3_index_bytes(dst)["device_bytes"]
        torch.cuda.synchronize()
        base = rb.rb3_device_peak(reset=True)
        a = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        a.record(st)
        rb.rb3_merge_opts(dst, src, opts, stream=st)
        e.record(st)
        torch.cuda.synchronize()
        res[name] = {"merge_ms": round(a.elapsed_time(e), 3), "index_bytes_before": before,
                     "index_bytes_after": rb.rb3_index_bytes(dst)["device_bytes"],
                     "peak_above_before_bytes": rb.rb3_device_peak() - base}
        src.free()
    n = rb.rb3_index_info(P)["n"]
    cp = torch.empty(n, dtype=torch.uint8, device="cuda")
    cr = torch.empty(n, dtype=torch.uint8, device="cuda")
    rb.rb3_export(P, codes=cp, stream=st)
    rb.rb3_export(R, codes=cr, stream=st)
    torch.cuda.synchronize()
    res["equal_output"] = bool(torch.equal(cp, cr))
    P.free()
    R.free()
    return res


def plain_vs_segmented(rb, torch, dev_batches, opts, st, ds):
    """Times the merge of batch 1 into batch 0 both ways (builds excluded)."""
    res = {}
    for form in (0, 1):
        base = rb.rb3_build_batch(*dev_batches[0], opts=opts, stream=st)
        src = rb.rb3_build_batch(*dev_batches[1], opts=opts, stream=st)
        o = dict(opts, merge_form=form)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        rb.rb3_merge_opts(base, src, o, stream=st)
        b.record(st)
        torch.cuda.synchronize()
        res["plain_ms" if form else "segmented_ms"] = round(a.elapsed_time(b), 3)
        if form == 0:
            ref = rb.rb3_export(base)
        else:
            res["equal_output"] = bool(np.array_equal(ref, rb.rb3_export(base)))
        base.free()
        src.free()
    res["speedup"] = round(res["plain_ms"] / res["segmented_ms"], 2)
    res["batch"] = "batch 1 (10 haplotypes, both strands) into batch 0"
    res["new_symbols"] = ds[1]
    return res


def locate_bench(rb, torch, S, args, st, dev, opts, batches, off, s=32):
    """Locate (Algorithm 2) on the same workload built with a sampled suffix
    array: the extra build time of the sample, and the SMEM hits of the
    benchmark queries located (the first row of every SMEM interval)."""
    ends = np.array([b for (_, b) in batches], dtype=np.int64)
    seq = torch.from_numpy(S.seq.copy()).to(dev)
    res = {"sa_sample": s}
    times = {}
    for rate in (0, s):
        o = dict(opts, sa_sample=rate)
        idx = rb.rb3_index_empty(o)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rb.rb3_append_batches(idx, seq, S.lens.copy(), ends, o, stream=st)
        torch.cuda.synchronize()
        times[rate] = (time.perf_counter() - t0) * 1e3
        if rate:
            Q = synth.mem_queries(S, nq=args.queries)
            q = torch.from_numpy(Q.q).to(dev)
            qoff = torch.from_numpy(Q.qoff).to(dev)
            cap = max(1 << 20, int(Q.qoff[-1]) // 16)
            recs = torch.empty(cap * 40, dtype=torch.uint8, device=dev)
            _, n = rb.rb3_mem_search(idx, q, qoff, 31, 1, out=recs, cap=cap, stream=st)
            rows = recs[:n * 40].view(n, 40)[:, 16:24].contiguous().view(torch.int64).flatten()
            out = torch.empty((n, 2), dtype=torch.int64, device=dev)
            rb.rb3_locate(idx, rows, out=out, stream=st)  # warm-up
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(st)
            rb.rb3_locate(idx, rows, out=out, stream=st)
            b.record(st)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            res.update({"rows": int(n), "ms": round(ms, 3), "value": round(n / (ms * 1e3), 2), "unit": "M rows/s",
                        "what": "the first row of every SMEM of the MEM-search queries"})
        idx.free()
    res["append"] = "all five batches appended to an empty index, ms"
    res["append_ms_without_sample"] = round(times[0], 1)
    res["append_ms_with_sample"] = round(times[s], 1)
    return res


def run_length_bench(rb, torch, S, idx, args, st, dev, chunk_len):
    """The finished index compressed to the run-length layout at a few span
    lengths: its device bytes against the plain index's, the compression time,
    and the MEM search of the benchmark queries on it (same outputs as on the
    plain index, checked on the device)."""
    Q = synth.mem_queries(S, nq=args.queries)
    q = torch.from_numpy(Q.q).to(dev)
    qoff = torch.from_numpy(Q.qoff).to(dev)
    bp = int(Q.qoff[-1])
    cap = max(1 << 20, bp // 16)
    o = {"search_form": 0, "chunk_len": int(chunk_len)}
    ref = torch.empty(cap * 40, dtype=torch.uint8, device=dev)
    _, n_ref = rb.rb3_mem_search_opts(idx, q, qoff, 31, 1, o, out=ref, cap=cap, stream=st)
    info = rb.rb3_index_info(idx)
    plain = rb.rb3_index_bytes(idx)["device_bytes"]
    res = {"plain_bytes": plain, "plain_occ_interval": info["occ_interval"], "spans": []}
    out = torch.empty(cap * 40, dtype=torch.uint8, device=dev)
    for span in (512, 1024, 2048, 4096, 16384):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        R = rb.rb3_index_compress(idx, span, stream=st)
        torch.cuda.synchronize()
        cms = (time.perf_counter() - t0) * 1e3
        nb = rb.rb3_index_bytes(R)
        _, n = rb.rb3_mem_search_opts(R, q, qoff, 31, 1, o, out=out, cap=cap, stream=st)  # warm-up
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        _, n = rb.rb3_mem_search_opts(R, q, qoff, 31, 1, o, out=out, cap=cap, stream=st)
        b.record(st)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        same = n == n_ref and bool(torch.equal(out[:n * 40], ref[:n_ref * 40]))
        res["spans"].append({"span": span, "runs": nb["runs"], "avg_run": round(info["n"] / max(1, nb["runs"]), 1),
                             "bytes": nb["device_bytes"], "bytes_per_symbol": round(nb["device_bytes"] / info["n"], 4),
                             "vs_plain": round(nb["device_bytes"] / plain, 4), "compress_ms": round(cms, 1),
                             "mem_search_value": round(bp / (ms * 1e3), 2), "mem_search_ms": round(ms, 3),
                             "equal_output": same})
        R.free()
    res["unit"] = "Mbp/s (mem_search_value)"
    return res


def diversity_kmers(S, k=51, n_kmers=20_000):
    """The diversity leg's queries: the n_kmers sliding k-mers of a window of
    one haplotype with 1% substitutions (a new sample), back to back."""
    g = synth.rng(synth.SEED_BASE + 77)
    off = S.offsets
    h = int(g.integers(0, len(S.lens)))
    st0 = int(off[h] + g.integers(0, max(1, S.lens[h] - (n_kmers + k))))
    win = S.seq[st0:st0 + n_kmers + k - 1].copy()
    win[win == 0] = 1
    sub = g.random(len(win)) < 0.01
    win[sub] = (win[sub] % 4) + 1
    nq = len(win) - k + 1
    starts = np.arange(nq, dtype=np.int64)
    q = win[starts[:, None] + np.arange(k)].reshape(-1).astype(np.uint8)
    qoff = np.arange(nq + 1, dtype=np.int64) * k
    return q, qoff


def diversity_bench(rb, torch, S, idx, st, dev, probe_g, k=51, n_kmers=20_000, W=25):
    """Local haplotype diversity of sliding k-mers of a new sample (a window
    of one haplotype with 1% substitutions), one k-mer per query, default
    scores, on the finished index: queries/s, and the kernel's rank-all reads
    per second against the random-read probe (each read is a dependent random
    32-byte access at D = 32)."""
    q, qoff = diversity_kmers(S, k, n_kmers)
    nq = len(qoff) - 1
    dq, doff = torch.from_numpy(q).to(dev), torch.from_numpy(qoff).to(dev)
    out = torch.empty((nq, W, 4), dtype=torch.int64, device=dev)
    n_out = torch.empty(nq, dtype=torch.int64, device=dev)
    res = {"workload": f"{nq} sliding {k}-mers of a haplotype window with 1% substitutions, scores a=1 b=3 q=5 e=2, "
                       f"W={W}, redundancy filter on, on the finished index", "unit": "queries/s"}
    try:
        rb.rb3_haplotype_diversity(idx, dq, doff, 1, 3, 5, 2, W, True, out=out, n_out=n_out, stream=st)  # warm-up
        torch.cuda.synchronize()
        rb.rb3_diversity_stats(reset=True)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        reps = 2
        a.record(st)
        for _ in range(reps):
            rb.rb3_haplotype_diversity(idx, dq, doff, 1, 3, 5, 2, W, True, out=out, n_out=n_out, stream=st)
        b.record(st)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / reps
        stats = rb.rb3_diversity_stats(reset=True)
        reads = stats["rank_reads"] / reps
        n = n_out.cpu().numpy()
        res.update({"value": round(nq / (ms * 1e-3), 1), "ms": round(ms, 3), "records_per_query": round(float(n.mean()), 2),
                    "queries_with_records": int((n > 0).sum()), "rank_reads_per_launch": int(reads),
                    "cells_per_launch": int(stats["cells"] / reps),
                    "rank_reads_G_per_s": round(reads / (ms * 1e-3) / 1e9, 3)})
        if probe_g:
            res["roofline"] = {"bound": "random_requests", "achieved": res["rank_reads_G_per_s"], "peak": probe_g,
                               "unit": "G req/s", "frac": round(res["rank_reads_G_per_s"] / probe_g, 4),
                               "what": "rank-all reads counted by the kernel over its CUDA-event time; ceiling: "
                                       "the random-read probe of the merge walk's roofline"}
    except (rb.RB3Error, RuntimeError) as e:  # a side leg: record the failure, keep the bench line
        res["error"] = f"{type(e).__name__}: {e}"
    return res


def bwasw_bench(rb, torch, S, idx, st, dev, nq=2000, L=150):
    """BWA-SW between query DAWGs and the finished index (Algorithm 5 with
    the query as a DAWG): nq queries of L bp from the haplotypes with 2%
    substitutions, default scores, W = 25; queries/s and records."""
    Q = synth.mem_queries(S, seed=synth.SEED_BASE + 79, nq=nq, median=L, sigma=0.0, lo=L, hi=L, sub=0.02,
                          random_frac=0.0)
    dq, doff = torch.from_numpy(Q.q).to(dev), torch.from_numpy(Q.qoff).to(dev)
    cap = nq * 2 * (L + 1) * 25
    out = torch.empty((cap, 7), dtype=torch.int64, device=dev)
    res = {"workload": f"{nq} queries of {L} bp from the haplotypes with 2% substitutions, scores a=1 b=3 q=5 e=2, "
                       "W=25, on the finished index", "unit": "queries/s"}
    try:
        n = rb.rb3_bwasw(idx, dq, doff, 1, 3, 5, 2, 25, cap=cap, out=out, stream=st)  # warm-up
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        n = rb.rb3_bwasw(idx, dq, doff, 1, 3, 5, 2, 25, cap=cap, out=out, stream=st)
        b.record(st)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        res.update({"value": round(nq / (ms * 1e-3), 1), "ms": round(ms, 3), "records": int(n),
                    "records_per_query": round(n / nq, 1)})
    except (rb.RB3Error, RuntimeError) as e:  # a side leg: record the failure, keep the bench line
        res["error"] = f"{type(e).__name__}: {e}"
    return res


def diversity_cpu_sample(S, window: int = 20_000, k: int = 51, nq: int = 300, W: int = 25):
    """The oracle's haplotype diversity on a bounded sample of the same
    workload: the double-strand BWT (naive sort, untimed) of the first
    `window` bp of every haplotype, and `nq` sliding k-mers of one haplotype's
    window with 1% substitutions, default scores; one thread."""
    import oracle
    off = S.offsets
    wins = [S.seq[off[h]:off[h] + min(window, S.lens[h])] for h in range(len(S.lens))]
    lens = np.array([len(w) for w in wins], dtype=np.int64)
    B = oracle.bwt(oracle.concat(np.concatenate(wins), lens, True))
    g = synth.rng(synth.SEED_BASE + 78)
    win = wins[int(g.integers(0, len(wins)))][:nq + k - 1].copy()
    win[win == 0] = 1
    sub = g.random(len(win)) < 0.01
    win[sub] = (win[sub] % 4) + 1
    n = len(win) - k + 1
    t = time.perf_counter()
    for i in range(n):
        oracle.haplotype_diversity(B, win[i:i + k], 1, 3, 5, 2, W=W)
    dt = time.perf_counter() - t
    return {"value": round(n / dt, 2), "unit": "queries/s", "cores": 1, "kind": "oracle",
            "sample": f"{n} sliding {k}-mers of one haplotype's first {window} bp with 1% substitutions against "
                      f"the oracle's double-strand BWT of the first {window} bp of all {len(wins)} haplotypes "
                      f"({len(B)} symbols): {dt:.2f} s"}


def mem_search(rb, torch, S, idx, args, st, dev, probe_g=None):
    Q = synth.mem_queries(S, nq=args.queries)
    q = torch.from_numpy(Q.q).to(dev)
    qoff = torch.from_numpy(Q.qoff).to(dev)
    bp = int(Q.qoff[-1])
    res = {"workload": f"{Q.nq} queries (lognormal len, median 150, sigma 1, clipped [31, 10000]; 90% haplotype "
                       "windows with 1% substitutions, 10% random), SMEMs >= 31 bp, min_occ 1, on the finished index",
           "query_bp": bp, "unit": "Mbp/s"}
    cap = max(1 << 20, bp // 16)
    out = torch.empty(cap * 40, dtype=torch.uint8, device=dev)
    # autotune the chunk length on the first 100k queries (untimed)
    ns = min(Q.nq, 100_000)
    best, tms = rb.rb3_tune_search(idx, q[:int(Q.qoff[ns])], qoff[:ns + 1], 31, 1, stream=st)
    res["autotune_chunk_len"] = int(best.chunk_len)
    res["autotune_hot_depth"] = int(best.hot_depth)
    for form, key, hot in ((0, "value", int(best.hot_depth)), (0, "no_hot_table_value", -1),
                           (2, "loops_value", 0), (1, "plain_value", 0)):
        o = {"search_form": form, "chunk_len": int(best.chunk_len), "hot_depth": hot}
        main = key == "value"
        reps = 2 if form == 0 else 1
        _, n = rb.rb3_mem_search_opts(idx, q, qoff, 31, 1, o, out=out, cap=cap, stream=st)  # warm-up
        torch.cuda.synchronize()
        if main:
            rb.rb3_search_stats(reset=True)
            rb.rb3_profile_reset()
            rb.rb3_profile_enable(True)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        for _ in range(reps):
            _, n = rb.rb3_mem_search_opts(idx, q, qoff, 31, 1, o, out=out, cap=cap, stream=st)
        b.record(st)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / reps
        res[key] = round(bp / (ms * 1e3), 2)
        res[key.replace("value", "ms")] = round(ms, 3)
        res["smems"] = int(n)
        if main:
            rb.rb3_profile_enable(False)
            kms = rb.rb3_profile_read().get("k.smem_steps", (ms * reps, reps, 0))[0] / reps
            ss = rb.rb3_search_stats(reset=True)
            reads, ext = ss["block_reads"] / reps, ss["extensions"] / reps
            rate = reads / (kms * 1e-3) / 1e9
            hbm, peak_kind = peaks()
            res["roofline"] = {
                "kernel": "k.smem_steps", "bound": "random_requests", "achieved": round(rate, 3),
                "peak": probe_g, "unit": "G req/s", "frac": round(rate / probe_g, 4) if probe_g else None,
                "kernel_ms": round(kms, 3), "extensions_per_base": round(ext / bp, 3),
                "block_reads_per_base": round(reads / bp, 3),
                "bytes_per_base": round(32 * reads / bp, 1),
                "hbm_frac": round(32 * reads / (kms * 1e-3) / 1e9 / hbm, 4), "hbm_peak_kind": peak_kind,
                "what": "Occ block reads (one 32-byte request each at D = 32; a hot-level table read counts "
                        "as one) counted by the kernel over its CUDA-event time; ceiling: the random-read probe "
                        "(32-byte dependent reads); hbm_frac: those bytes per second against the copy peak"}
    res["speedup_vs_plain"] = round(res["value"] / res["plain_value"], 2)
    return res


def _serve_trace(rb, srv, arr, Q):
    """Open-loop replay on the library's native submitter: each request
    submitted at its arrival time; latency = completion time - scheduled
    arrival time."""
    done, batch = rb.rb3_server_replay(srv, Q.q, Q.qoff, arr)
    lat = (done - arr) * 1e3
    bp = int(Q.qoff[-1])
    ws = rb.rb3_server_stats(srv)
    busy = max(1, ws["gather_ns"] + ws["search_ns"] + ws["publish_ns"])
    return {"p50_ms": round(float(np.percentile(lat, 50)), 3), "p99_ms": round(float(np.percentile(lat, 99)), 3),
            "Mbp_per_s": round(bp / float(done.max()) / 1e6, 1), "mean_batch": round(float(batch.mean()), 2),
            "slot_time": {"gather": round(ws["gather_ns"] / busy, 3), "search": round(ws["search_ns"] / busy, 3),
                          "publish": round(ws["publish_ns"] / busy, 3),
                          "search_ms_per_batch": round(ws["search_ns"] / 1e6 / max(1, ws["batches"]), 3)}}


SERVE_RATES = (2000, 5000, 10000, 20000, 50000, 100000, 200000, 500000, 1000000)


def served(rb, S, idx, index_desc, rates=SERVE_RATES, n_cap=20000, unbatched_max_rate=10000):
    """The served workload's request law (query lengths log-uniform in [100,
    100000] bp with 0.1-5% substitutions) replayed as Poisson arrivals at each
    rate, up to and past saturation (min(rate x 1 s, 20,000) requests of one
    request set per rate): continuous batching (4 slots) with the step-machine
    search, the same with the plain one-query-per-thread kernel (equal output),
    and no batching (one request per micro-batch, one slot) at the low rates."""
    res = {"index": index_desc, "requests": "Poisson arrivals; lengths log-uniform 100 bp-100 kb; "
                                            "0.1-5% substitutions; SMEMs >= 31 bp", "rates": {}}
    _, Qall = synth.served_requests(S, rate=2000.0, n_req=n_cap)
    forms = (("batched", dict(slots=4)), ("batched_plain_kernel", dict(slots=4, search_form=1)),
             ("unbatched", dict(slots=1, max_batch_requests=1)))
    for rate in rates:
        n = int(min(n_cap, max(1000, rate)))
        Q = Qall.subset(np.arange(n))
        arr = np.cumsum(synth.rng(synth.SEED_BASE + 40 + rate).exponential(1.0 / rate, size=n))
        row = {"n_requests": n, "offered_Mbp_per_s": round(float(Q.qoff[-1]) / arr[-1] / 1e6, 1)}
        for name, kw in forms:
            if name == "unbatched" and rate > unbatched_max_rate:
                continue
            srv = rb.rb3_server_create(idx, **kw)
            row[name] = _serve_trace(rb, srv, arr, Q)
            srv.close()
        res["rates"][str(rate)] = row
    return res


def uneven_bench(rb, torch, st, dev, n_genomes):
    """The uneven-genome workload (2,000 bacterial-like genomes in 20 clusters,
    lognormal lengths, 1% substitutions, 0.5% N-runs; batches of 64 genomes),
    its first n_genomes: rb3_tune_build picks the Occ interval, segment length
    and seed cap on batches 0-1 (untimed); then every batch is appended to an
    empty index through rb3_append_batches (timed, CUDA events), Msym/s."""
    S = synth.uneven(n_genomes=n_genomes)
    ends = np.array([b for (_, b) in S.batches], dtype=np.int64)
    seq = torch.from_numpy(S.seq).to(dev)
    res = {"workload": f"uneven genomes: the first {n_genomes} of 2000 (20 clusters, lognormal median 3 Mb, "
                       "1% substitutions, 0.5% N-runs 10-100), batches of 64, both strands",
           "genomes": n_genomes, "batches": len(ends), "symbols": S.ds_symbols()}
    if len(ends) < 2:
        res["error"] = "needs two batches"
        return res
    t = time.perf_counter()
    best, table = rb.rb3_tune_build(seq, S.lens, ends, stream=st)
    res["autotune"] = {"occ_interval": int(best.occ_interval), "seg_len": int(best.seg_len),
                       "seed_cap": int(best.seed_cap), "walk_ctas_per_sm": int(best.walk_ctas_per_sm) or 8,
                       "candidates": [{"D": d, "build_merge_ms": round(ms, 2), "index_mib": round(mb, 1)}
                                      for d, ms, mb in table],
                       "tune_s": round(time.perf_counter() - t, 2),
                       "what": "batch 1 built and merged into batch 0 at each D; the fastest whose projected "
                               "index fits (no budget given)"}
    idx = rb.rb3_index_empty(best)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(st)
    rb.rb3_append_batches(idx, seq, S.lens, ends, best, stream=st)
    b.record(st)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    info = rb.rb3_index_info(idx)
    res.update({"value": round(info["n"] / (ms * 1e3), 1), "unit": "Msym/s", "ms": round(ms, 1),
                "index_symbols": info["n"], "index_bytes": rb.rb3_index_bytes(idx)["device_bytes"]})
    idx.free()
    return res


def served_full(rb, torch, st, dev, opts):
    """The served workload on its own index: 20 haplotypes of a 150 Mb founder,
    built through rb3_append_batches in batches of 4 haplotypes."""
    S = synth.served_index_strings()
    off = S.offsets
    seq = torch.from_numpy(S.seq).to(dev)
    idx = rb.rb3_index_empty(opts)
    ends = np.array([b for (_, b) in S.batches], dtype=np.int64)
    t = time.perf_counter()
    rb.rb3_append_batches(idx, seq, S.lens.copy(), ends, opts, stream=st)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t
    del seq
    info = rb.rb3_index_info(idx)
    out = {"index_symbols": info["n"], "build_s": round(build_s, 2),
           "build_Msym_per_s": round(info["n"] / build_s / 1e6, 1),
           "served": served(rb, S, idx, "served index: 20 haplotypes of a 150 Mb founder (~6 Gsym)")}
    idx.free()
    return out


# ---------------------------------------------------------------------------
# CPU oracle: bounded sample of the same workload
# ---------------------------------------------------------------------------
def oracle_sample_inputs(S, window: int):
    """Windows of haplotype 0 (batch 0) and haplotype 10 (batch 1)."""
    off = S.offsets
    a = S.seq[off[0]:off[0] + min(window, S.lens[0])]
    b = S.seq[off[10]:off[10] + min(window, S.lens[10])]
    return a.copy(), b.copy()


def oracle_step(oracle, B1, b):
    """One oracle step: naive-sort BWT of the new batch (both strands) + Algorithm 1 merge."""
    T2 = oracle.concat(b, np.array([len(b)]), True)
    t = time.perf_counter()
    B2 = oracle.bwt(T2)
    M = oracle.merge(B1, B2, nthreads=2)
    dt = time.perf_counter() - t
    return len(T2), dt, M


def cpu_sample(S, window: int = 5_000_000):
    import oracle
    a, b = oracle_sample_inputs(S, window)
    B1 = oracle.bwt(oracle.concat(a, np.array([len(a)]), True))
    n2, dt, _ = oracle_step(oracle, B1, b)
    return {"value": round(n2 / dt / 1e6, 4), "unit": "Msym/s", "cores": 2, "kind": "oracle",
            "host_cores": os.cpu_count(), "b1_symbols": int(len(B1)), "b2_symbols": int(n2),
            "b1_note": "the workload's steps merge 100 Msym batches into 100-400 Msym indexes; this sample's index "
                       "is one haplotype window (10 Msym), so its rank table is far smaller",
            "sample": f"build (naive suffix sort, 1 thread) of the double-strand BWT of a {len(b)} bp window of "
                      f"haplotype 10 and Algorithm 1 merge (2 walks, 2 threads) into that of haplotype 0's window: "
                      f"{n2} new symbols in {dt:.2f} s"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    S = synth.pangenome(founder_len=int(5_000_000 * args.scale), n_hap=50, batch=10)
    a, b = oracle_sample_inputs(S, 5_000_000)
    B1 = oracle.bwt(oracle.concat(a, np.array([len(a)]), True))
    for _ in range(args.warmup):
        oracle_step(oracle, B1, b)
    tot_n, tot_t = 0, 0.0
    for _ in range(args.steps):
        n2, dt, _ = oracle_step(oracle, B1, b)
        tot_n += n2
        tot_t += dt
    v = tot_n / tot_t / 1e6
    sample = (f"each step: naive-sort double-strand BWT of a {len(b)} bp window of haplotype 10 + Algorithm 1 "
              f"merge into haplotype 0's window ({tot_n // args.steps} new symbols)")
    out = {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "Msym/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(tot_t / args.steps * 1e3, 1),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "parallelism": "CPU oracle, host cores"},
           "cpu_baseline": {"value": round(v, 4), "unit": "Msym/s", "cores": 2, "kind": "oracle", "sample": sample},
           "e2e": {"value": round(v, 4), "unit": "Msym/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    rank, world, local_rank = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_rb3(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
