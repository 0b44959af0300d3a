#!/usr/bin/env python
"""Benchmark of the k-mismatch FM-index search (the BWT phase of MICA, Section 2).

Workload: the 64 Mbp synthetic repeat genome (i.i.d. base, 5% copies of
1-10 kbp at 1% divergence, 1% tandem arrays) and 1,000,000 reads of 150 bp
with 1% substitution error, k <= 2 on both strands, at most 1000 listed hits
per read (exact totals).  One step = one batch of 1M reads through the whole
path (seed lookups, backtracking, counting and capping, LF-walk location,
per-read sort) with the reads already in HBM; the index is built once.

At one GPU the line also carries two more workloads, each its own sub-object
with its own roofline:
  "uneven": 1M reads of 50/100/150/250 bp with k in 0..3 (30% from repeats)
            on the same genome: one persistent launch vs one plain launch per
            length class and one plain launch;
  "human":  a 3.1 Gbp synthetic genome (about 45% repeats) resident in HBM and
            one batch of 1M read pairs (2M mates of 150 bp, k <= 2 per mate):
            persistent vs plain, against the HBM random-gather ceiling.

  python bench.py [--gpus N --steps K --warmup W]       our CUDA path (N replicas)
  python bench.py --impl reference [...]                the CPU oracle, timed
  python bench.py --workload uneven|human|serve         one workload on its own

Prints one JSON line on rank 0.
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

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "150bp reads/s aligned (k<=2 FM search) batched vs plain kernel; p99 latency"
WORKLOAD = "64 Mbp repeat genome, 1M x 150 bp reads (1% substitutions), k<=2 both strands, cap 1000"
HIT_CAP = 1000
PAIR_WINDOW = (300, 700)   # fragment lengths of the human-scale pairs: Normal(500, 50) clipped to this
L2_FLUSH_BYTES = 512 << 20
PROFILE = os.path.join(ROOT, "profiles", "k_persistent_64m_1m150.txt")
PROFILE_HUMAN = os.path.join(ROOT, "profiles", "k_persistent_3g_human2m.txt")
SEARCH_CU = os.path.join(ROOT, "paper_1402_4876_gb300", "csrc", "search.cu")
BIDIR_CU = os.path.join(ROOT, "paper_1402_4876_gb300", "csrc", "bidir.cu")
PROFILE_BIDIR = os.path.join(ROOT, "profiles", "k_bidir_64m_1m150.txt")
PROFILE_BIDIR_HUMAN = os.path.join(ROOT, "profiles", "k_bidir_3g_human2m.txt")
KERNEL_NAMES = {"bidirectional": "k_bidir", "persistent": "k_lower_bounds + k_persistent"}
KERNEL_LABEL = {"bidirectional": "bidirectional warp-pool (one persistent launch)",
                "persistent": "one-directional persistent warp-pool"}
SEARCH_LABEL = {"bidirectional": "k + 1 pieces, one search per leftmost exact piece over the genome's and the "
                                 "reversed genome's index (same result as exhaustive backtracking)",
                "persistent": "exhaustive backtracking from the read's end, pruned by mismatch lower bounds "
                              "(same result as unpruned)"}
ALG_LABEL = {"bidirectional": "32 B x occurrence blocks read + 16 B x seeds (two table entries in each of two "
                              "tables) + the packed reads once + 16 B x leaf intervals + the bytes of the text "
                              "checks (4 B of SA and the window's text words per check, 4 B of ISA per leaf)",
             "persistent": "32 B x occurrence blocks read (search and lower-bound pass) + 8 B x seeds + the "
                           "packed reads twice + 16 B x leaf intervals"}


def search_alg_bytes(kernel: str, st: dict, read_bytes: int) -> int:
    """Algorithmic bytes of one search step from the on-device work counters."""
    if kernel == "bidirectional":
        return (32 * st["rank_blocks"] + 16 * st["seeds"] + read_bytes + 16 * st["intervals"] +
                st.get("verify_bytes", 0))
    return 32 * st["rank_blocks"] + 8 * st["seeds"] + 2 * read_bytes + 16 * st["intervals"]


def gather_floor(kernel: str, st: dict, read_bytes: int, index_gbs: float, text_gbs: float, copy_gbs: float):
    """The least time a search step's memory accesses can take at the measured
    ceilings: every 32-byte sector it gathers from the index (occurrence
    blocks, one q-mer table sector per table and seed, leaf writes) at the
    random-gather rate of the level the index lives in (L2 when it fits, else
    HBM), every sector of the text checks (SA, ISA, text windows: HBM) at the
    HBM random-gather rate, and the packed reads streamed at copy bandwidth.
    Returns (seconds, parts in ms)."""
    seed_sectors = (2 if kernel == "bidirectional" else 1) * st["seeds"]
    index_sectors = st["rank_blocks"] + seed_sectors + (st["intervals"] + 1) // 2
    t_index = index_sectors * 32 / (index_gbs * 1e9)
    t_text = st.get("verify_sectors", 0) * 32 / (text_gbs * 1e9)
    t_reads = (read_bytes if kernel == "bidirectional" else 2 * read_bytes) / (copy_gbs * 1e9)
    parts = {"index_gathers_ms": round(t_index * 1e3, 4), "text_check_gathers_ms": round(t_text * 1e3, 4),
             "read_stream_ms": round(t_reads * 1e3, 4), "index_sectors": int(index_sectors),
             "text_check_sectors": int(st.get("verify_sectors", 0))}
    return t_index + t_text + t_reads, parts


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--reads", type=int, default=1_000_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--kernel", default="bidirectional", choices=["bidirectional", "persistent"],
                    help="the batched kernel timed for the headline (the other is timed beside it)")
    ap.add_argument("--no-uneven", action="store_true", help="leave the uneven-batch leg out of the default line")
    ap.add_argument("--no-human", action="store_true", help="leave the human-scale leg out of the default line")
    ap.add_argument("--human-pairs", type=int, default=1_000_000, help="default line: pairs of the human-scale leg")
    ap.add_argument("--workload", default="repeats64m", choices=["repeats64m", "uneven", "human", "serve"],
                    help="repeats64m: the headline; uneven: mixed lengths and budgets; human: 3.1 Gbp genome, "
                         "10M read pairs; serve: Poisson requests on a resident index")
    ap.add_argument("--pairs", type=int, default=10_000_000, help="human: read pairs")
    ap.add_argument("--genome-bp", type=int, default=synth.HUMAN_LEN, help="human/serve: genome length")
    ap.add_argument("--serve-requests", type=int, default=200, help="serve: requests per load level")
    ap.add_argument("--serve-max-size", type=int, default=1_000_000, help="serve: largest request (reads)")
    ap.add_argument("--serve-tick", type=int, default=1 << 20, help="serve: reads per search launch")
    ap.add_argument("--serve-chunk", type=int, default=1 << 18, help="serve: largest piece of a request per launch")
    ap.add_argument("--serve-kernel", default="bidirectional", help="serve: search kernel")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


# ---- replicas: every GPU holds its own index and aligns its own batch; the
# ranks meet only for a barrier and the max-over-ranks time (gloo, host) ----

def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seed(rank: int) -> int:
    """Each replica aligns its own batch: reads drawn with a per-rank seed."""
    return synth.SEED_READS_64M + rank


def whole_job_rate(reads_per_rank: int, world: int, steps: int, max_ms: float) -> float:
    """Units all ranks processed divided by the slowest rank's time."""
    return world * reads_per_rank * steps / (max_ms / 1e3)


def cpu_info():
    model = ""
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    if not model:
        try:
            model = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
            model = next((l.split(":", 1)[1].strip() for l in model.splitlines() if "Model name" in l), "")
        except Exception:
            model = ""
    return os.cpu_count() or 1, model


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = os.path.join("/tmp", f"mica_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        sm, mx, reasons = [], [], set()
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                for name, val in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                                      "sw_power_cap"), f[5:9]):
                    if val.lower() == "active":
                        reasons.add(name)
        except OSError:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0}, "fallback"


def profile_traffic(kernel_src: str, profile: str = PROFILE, key: str = "dram_bytes_per_launch_scaled"):
    """dram bytes per launch of the search step from a committed ncu summary,
    or None when the kernel source changed since the capture."""
    try:
        vals = {}
        for line in open(profile):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
        sha = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()[:16]
        if sha not in (vals.get("kernel_src_sha256_16"), vals.get("search_cu_sha256_16")):
            return None
        return float(vals[key])
    except Exception:
        return None


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------

def make_workload(n_reads: int, rank: int):
    g = synth.genome_64m()
    reads = synth.reads_64m(g, n=n_reads, seed=replica_seed(rank))
    return g, reads


def gather_ceilings(mica, idx, device: int, kernel: str = "bidirectional") -> dict:
    """Random 32-byte gather ceilings measured after the timed region: one
    over a buffer the size of the search's hot index arrays (occurrence
    blocks + q-mer tables, of both directions for the bidirectional kernel:
    the same L2/HBM mix as the search), one over 1.5 GiB (HBM)."""
    info = idx.info()
    hot = info["occ_bytes"] + info["table_bytes"]
    if kernel == "bidirectional":
        hot += info["rev_occ_bytes"] + info["rev_table_bytes"]
    hot = max(1 << 20, (hot + 31) // 32 * 32)
    a = mica.gather_ceiling(hot, 32, loads=1 << 27, repeats=3, device=device)
    b = mica.gather_ceiling(3 << 29, 32, loads=1 << 27, repeats=3, device=device)
    return {"load_bytes": 32, "index_sized_bytes": hot, "index_sized_gbs": round(a["gbs"], 1),
            "hbm_bytes": 3 << 29, "hbm_gbs": round(b["gbs"], 1),
            "what": "mica_gather_ceiling: independent random 32 B loads, full occupancy"}


def run_ours(args):
    import torch
    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    import paper_1402_4876_gb300 as mica

    g, b = make_workload(args.reads, rank)
    t0 = time.perf_counter()
    idx = mica.Index.build(synth.to_acgt_bytes(g.codes), kmer_q=12, sa_sample=16, device=local)
    build_s = time.perf_counter() - t0

    dev = torch.device("cuda", local)
    d_words = torch.from_numpy(b.words.view(np.int32)).to(dev)
    d_off = torch.from_numpy(b.word_off.view(np.int64)).to(dev)
    d_len = torch.from_numpy(b.lengths.view(np.int16)).to(dev)
    d_k = torch.from_numpy(b.k).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)


    def device_steps(kernel: str, steps: int, warmup: int, prune: bool = True, report: str = "all"):
        for _ in range(warmup):
            idx.align_device(d_words, d_off, d_len, d_k, b.n, hit_cap=HIT_CAP, kernel=kernel, stream=stream,
                             prune=prune, report=report)
        ms, kms, stats = [], [], []
        barrier(world)
        torch.cuda.synchronize(dev)
        for _ in range(steps):
            flush.fill_(rank + len(ms))                      # evict L2 between timed steps
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = idx.align_device(d_words, d_off, d_len, d_k, b.n, hit_cap=HIT_CAP, kernel=kernel,
                                 stream=stream, prune=prune, report=report)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            st = idx.stats()
            kms.append(st["kernel_ms"])
            stats.append(st)
        torch.cuda.synchronize(dev)
        barrier(world)
        return ms, kms, stats, r

    with ClockSampler(local) as clk:
        ms, kms, stats, dres = device_steps(args.kernel, args.steps, args.warmup)
    clocks = clk.summary()
    total_ms = max_over_ranks(sum(ms), world)
    value = whole_job_rate(b.n, world, args.steps, total_ms)
    n_hits = dres.n_hits

    out = {
        "metric": METRIC, "value": round(value, 1), "unit": "reads/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic (seeded generator; the paper's YH/1000 Genomes data are not available)",
        "config": {"workload": WORKLOAD, "genome_bp": g.n, "reads_per_gpu": b.n, "read_len": 150, "k": 2,
                   "hit_cap": HIT_CAP, "kernel": KERNEL_LABEL[args.kernel],
                   "index": "q=12 tables of the genome and its reversal, 32 B bit-plane occurrence blocks of both, "
                            "SA 1/16",
                   "search": SEARCH_LABEL[args.kernel],
                   "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write)",
                   "parallelism": f"replicas x{world} (index per GPU, reads sharded, no collective)"},
        "latency_ms": {"p50": round(float(np.percentile(ms, 50)), 3), "p99": round(float(np.percentile(ms, 99)), 3),
                       "what": "per-batch (1M reads) device latency over the timed steps"},
        "index_build_s": round(build_s, 3),
        "hits_per_step": int(n_hits),
    }
    st = stats[-1]
    out["work_per_step"] = {k: int(st[k]) for k in ("seeds", "nodes", "rank_blocks", "intervals", "located",
                                                    "lf_steps", "spills", "lb_steps", "lb_dead_tasks",
                                                    "verified", "verify_bytes", "verify_sectors", "warp_rounds",
                                                    "grid_ctas")}
    if st["warp_rounds"]:
        out["work_per_step"]["lanes_per_round"] = round(
            (st["nodes"] + st["seeds"] + st["verified"]) / st["warp_rounds"], 2)
    out["gpu_launches"] = int(sum(s["launches"] for s in stats))
    out["graph_replays"] = int(sum(s["graph_replays"] for s in stats))

    # roofline of the dominant kernel(s) of the search step.  The 64 Mbp index
    # (occurrence blocks and q-mer tables, under 129 MB) stays in L2, so the
    # step is bound by dependent random 32-byte gathers from L2, not by HBM:
    # its ceiling is the measured random-gather rate over a buffer of the
    # index's size, taken in this run.
    peaks, src = measured_peaks()
    kernel_s = statistics.mean(kms) / 1e3
    read_bytes = 4 * int(np.sum((b.lengths.astype(np.int64) + 15) // 16))
    alg_bytes = search_alg_bytes(args.kernel, st, read_bytes)
    achieved = alg_bytes / kernel_s / 1e9
    traffic = profile_traffic(SEARCH_CU if args.kernel == "persistent" else BIDIR_CU,
                              PROFILE if args.kernel == "persistent" else PROFILE_BIDIR)
    ceil = gather_ceilings(mica, idx, local, args.kernel)
    gc_idx = ceil["index_sized_gbs"]
    t_floor, floor_parts = gather_floor(args.kernel, st, read_bytes, gc_idx, ceil["hbm_gbs"], peaks["hbm_gbs"])
    peak = alg_bytes / t_floor / 1e9
    out["roofline"] = {"bound": "random_gather_l2_and_hbm", "achieved": round(achieved, 1), "peak": round(peak, 1),
                       "unit": "GB/s", "frac": round(t_floor / kernel_s, 4), "traffic": traffic,
                       "kernel": KERNEL_NAMES[args.kernel] + " (one search step)",
                       "kernel_ms": round(kernel_s * 1e3, 3),
                       "alg_bytes_per_launch": int(alg_bytes),
                       "alg_bytes_what": ALG_LABEL[args.kernel],
                       "peak_source": "the step's algorithmic bytes / its gather floor: the least time its sectors "
                                      "take at the random-gather ceilings measured in this run (index gathers at "
                                      "the rate over an index-sized buffer, which stays in L2; text-check gathers "
                                      "at the rate over 1.5 GiB, HBM; reads at the copy bandwidth); frac = floor / "
                                      "kernel time",
                       "floor_ms": round(t_floor * 1e3, 4), "floor_parts": floor_parts,
                       "frac_of_index_gather_ceiling": round(achieved / gc_idx, 4) if gc_idx else None,
                       "hbm_copy_peak": peaks["hbm_gbs"],
                       "frac_of_hbm_copy": round(achieved / peaks["hbm_gbs"], 4),
                       "hbm_copy_peak_source": f"{src} hbm_gbs (MEASURED_PEAKS.json, copy bandwidth)",
                       "gather_ceiling": ceil,
                       "note": "the index stays in L2 (DRAM traffic of the step is a fraction of its algorithmic "
                               "bytes); the kernel is latency-bound on chains of dependent gathers"}
    out["clocks"] = clocks
    out["rank_blocks_per_s"] = round(st["rank_blocks"] / kernel_s, 1)
    out["mbp_per_s"] = round(value * float(np.mean(b.lengths)) / 1e6, 1)   # bases of reads aligned

    # the other batched kernel on the same batch
    other = "persistent" if args.kernel == "bidirectional" else "bidirectional"
    oms, okms, ostats, _ = device_steps(other, max(1, min(args.steps, 5)), 1)
    ototal = max_over_ranks(sum(oms), world)
    oval = whole_job_rate(b.n, world, len(oms), ototal)
    ost = ostats[-1]
    oalg = search_alg_bytes(other, ost, read_bytes)
    out[other] = {"value": round(oval, 1), "unit": "reads/s", "ms_per_step": round(ototal / len(oms), 3),
                  "kernel_ms": round(statistics.mean(okms), 3), "kernel": KERNEL_NAMES[other],
                  "search": SEARCH_LABEL[other], "nodes": int(ost["nodes"]), "seeds": int(ost["seeds"]),
                  "rank_blocks": int(ost["rank_blocks"]),
                  "roofline_frac": round(gather_floor(other, ost, read_bytes,
                                                      gather_ceilings(mica, idx, local, other)["index_sized_gbs"],
                                                      ceil["hbm_gbs"], peaks["hbm_gbs"])[0]
                                         / (statistics.mean(okms) / 1e3), 4),
                  f"{args.kernel}_over_{other}": round(value / oval, 3)}

    if not args.no_plain:
        # the same exhaustive search without lower-bound pruning (same result, more work)
        ums, ukms, ustats, _ = device_steps("persistent", max(1, min(args.steps, 3)), 1, prune=False)
        utotal = max_over_ranks(sum(ums), world)
        uval = whole_job_rate(b.n, world, len(ums), utotal)
        out["unpruned"] = {"value": round(uval, 1), "unit": "reads/s", "ms_per_step": round(utotal / len(ums), 3),
                           "kernel_ms": round(statistics.mean(ukms), 3), "nodes": int(ustats[-1]["nodes"]),
                           "seeds": int(ustats[-1]["seeds"]),
                           "pruned_over_unpruned": round((value if args.kernel == "persistent" else oval) / uval, 3),
                           "what": "the one-directional persistent search without lower-bound pruning"}
        # best-stratum reporting (iterative deepening over the mismatch budget)
        bms, bkms, bstats, _ = device_steps("persistent", max(1, min(args.steps, 3)), 1, report="best_stratum")
        btotal = max_over_ranks(sum(bms), world)
        out["best_stratum"] = {"value": round(whole_job_rate(b.n, world, len(bms), btotal), 1), "unit": "reads/s",
                               "ms_per_step": round(btotal / len(bms), 3),
                               "kernel_ms": round(statistics.mean(bkms), 3), "nodes": int(bstats[-1]["nodes"]),
                               "seeds": int(bstats[-1]["seeds"]),
                               "what": "report = best stratum: each read's placements with its smallest d "
                                       "(one-directional persistent kernel, deepening the budget pass by pass)"}
        pms, pkms, pstats, _ = device_steps("plain", max(1, min(args.steps, 3)), 1)
        ptotal = max_over_ranks(sum(pms), world)
        pval = whole_job_rate(b.n, world, len(pms), ptotal)
        out["plain"] = {"value": round(pval, 1), "unit": "reads/s", "ms_per_step": round(ptotal / len(pms), 3),
                        "kernel_ms": round(statistics.mean(pkms), 3),
                        "batched_over_plain": round(value / pval, 3),
                        "what": "one (read, strand) task per thread, lower-bound pruning, device re-queue"}

    if not args.no_e2e:
        # end to end through the public host-buffer API: every step copies its
        # batch in from pinned host memory and its result out (mica_align_submit /
        # mica_align_collect: while one batch searches, the next one's copies and
        # host checks run and the previous one's result comes back)
        pin = lambda a: torch.from_numpy(a).pin_memory().numpy()
        hw, ho, hl, hk = pin(b.words), pin(b.word_off), pin(b.lengths), pin(b.k)

        def stream_steps(count):
            prev, res = None, None
            for _ in range(count):
                t = idx.submit(hw, ho, hl, hk, hit_cap=HIT_CAP, kernel=args.kernel)
                if prev is not None:
                    res = idx.collect(prev)
                prev = t
            return idx.collect(prev)

        stream_steps(max(3, args.warmup))      # both slots capture their launch sequence
        barrier(world)
        e2e_steps = max(2, min(args.steps, 10))
        t = time.perf_counter()
        res = stream_steps(e2e_steps)
        el = max_over_ranks(time.perf_counter() - t, world)
        h2d = hw.nbytes + ho.nbytes + hl.nbytes + hk.nbytes
        d2h = res.total.nbytes + res.offsets.nbytes + res.hits.nbytes
        out["e2e"] = {"value": round(world * b.n * e2e_steps / el, 1), "unit": "reads/s",
                      "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                      "steps": e2e_steps,
                      "api": "mica_align_submit / mica_align_collect (host buffers: each step copies its pinned "
                             "input in and its result out; two batches in flight)",
                      "kernel": KERNEL_LABEL[args.kernel]}
        # the one-call form (mica_align_batch: copies, search and result in series)
        res = None
        for _ in range(max(2, args.warmup)):
            res = idx.align(hw, ho, hl, hk, hit_cap=HIT_CAP, kernel=args.kernel, stream=stream)
        barrier(world)
        one_steps = max(1, min(args.steps, 5))
        t = time.perf_counter()
        for _ in range(one_steps):
            res = idx.align(hw, ho, hl, hk, hit_cap=HIT_CAP, kernel=args.kernel, stream=stream)
        torch.cuda.synchronize(dev)
        el1 = max_over_ranks(time.perf_counter() - t, world)
        out["e2e"]["one_call"] = {"value": round(world * b.n * one_steps / el1, 1), "unit": "reads/s",
                                  "api": "mica_align_batch (copies in, search, result out, in series)"}

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(g, b)

    # the other workloads, one GPU only (replica runs time the headline alone)
    if world == 1:
        if not args.no_uneven:
            out["uneven"] = uneven_leg(mica, idx, g, args.reads, max(1, min(args.steps, 3)), 1, stream, flush,
                                       headline=args.kernel)
        idx.free()
        if not args.no_human:
            out["human"] = human_leg(mica, dev, stream, args.human_pairs, synth.HUMAN_LEN,
                                     steps=max(1, min(args.steps, 2)), plain=not args.no_plain,
                                     headline=args.kernel)

    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# other workloads (one GPU; printed as one JSON line each)
# ---------------------------------------------------------------------------

def _device_batch(b, dev):
    import torch
    return (torch.from_numpy(b.words.view(np.int32)).to(dev), torch.from_numpy(b.word_off.view(np.int64)).to(dev),
            torch.from_numpy(b.lengths.view(np.int16)).to(dev), torch.from_numpy(b.k).to(dev))


def _time_kernel(idx, d, n, kernel, steps, warmup, stream, flush=None):
    import torch
    for _ in range(warmup):
        idx.align_device(*d, n, hit_cap=HIT_CAP, kernel=kernel, stream=stream)
    ms, kms, st = [], [], None
    for _ in range(steps):
        if flush is not None:
            flush.fill_(len(ms))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = idx.align_device(*d, n, hit_cap=HIT_CAP, kernel=kernel, stream=stream)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        st = idx.stats()
        kms.append(st["kernel_ms"])
    return ms, kms, st, r


def uneven_leg(mica, idx, g, n_reads, steps, warmup, stream, flush, headline="bidirectional") -> dict:
    """Batched uneven: n_reads reads of 50/100/150/250 bp with k in 0..3 (30%
    from planted repeats) on the 64 Mbp repeat genome; one launch of each
    batched kernel (the bidirectional and the one-directional persistent one,
    autotuned shape) vs one plain launch per length class (autotuned block
    sizes) and one plain launch."""
    import torch
    dev = torch.device("cuda", 0)
    b = synth.reads_uneven(g, n=n_reads)
    tune = idx.autotune(b.subset(np.arange(0, b.n, max(1, b.n // 20000))), hit_cap=HIT_CAP, repeats=1)
    d = _device_batch(b, dev)
    out = {"workload": f"64 Mbp repeat genome, {b.n} reads, lengths uniform in {{50,100,150,250}}, "
                       "k uniform in 0..3, 30% from repeats, cap 1000",
           "unit": "reads/s", "steps": steps, "warmup": warmup, "tuning": tune,
           "l2": "flushed between timed steps"}
    for kernel in ("bidirectional", "persistent", "plain_by_length", "plain"):
        reps = steps if kernel in ("bidirectional", "persistent") else 1
        ms, kms, st, r = _time_kernel(idx, d, b.n, kernel, reps, warmup, stream, flush)
        out[kernel] = {"value": round(b.n * len(ms) / (sum(ms) / 1e3), 1), "ms_per_step": round(statistics.mean(ms), 3),
                       "kernel_ms": round(statistics.mean(kms), 3), "launches": int(st["launches"]),
                       "nodes": int(st["nodes"]), "seeds": int(st["seeds"]), "rank_blocks": int(st["rank_blocks"]),
                       "intervals": int(st["intervals"]), "retries": int(st["retries"]), "hits": int(r.n_hits),
                       "verified": int(st["verified"]), "verify_bytes": int(st["verify_bytes"]),
                       "verify_sectors": int(st["verify_sectors"])}
    h = out[headline]
    out["value"] = h["value"]
    out["kernel"] = KERNEL_LABEL[headline]
    for base in ("plain_by_length", "plain", "persistent", "bidirectional"):
        if base != headline:
            out[f"{headline}_over_{base}"] = round(h["value"] / out[base]["value"], 3)
    read_bytes = 4 * int(np.sum((b.lengths.astype(np.int64) + 15) // 16))
    alg = search_alg_bytes(headline, h, read_bytes)
    info = idx.info()
    hot = info["occ_bytes"] + info["table_bytes"] + info["rev_occ_bytes"] + info["rev_table_bytes"]
    ceil = mica.gather_ceiling(max(1 << 20, (hot + 31) // 32 * 32), 32, loads=1 << 27, repeats=3)
    hbm = mica.gather_ceiling(3 << 29, 32, loads=1 << 27, repeats=3)
    peaks, _ = measured_peaks()
    ach = alg / (h["kernel_ms"] / 1e3) / 1e9
    t_floor, parts = gather_floor(headline, h, read_bytes, ceil["gbs"], hbm["gbs"], peaks["hbm_gbs"])
    out["roofline"] = {"bound": "random_gather_l2_and_hbm", "achieved": round(ach, 1),
                       "peak": round(alg / t_floor / 1e9, 1), "unit": "GB/s",
                       "frac": round(t_floor / (h["kernel_ms"] / 1e3), 4), "kernel": KERNEL_NAMES[headline],
                       "alg_bytes_per_launch": int(alg), "alg_bytes_what": ALG_LABEL[headline],
                       "floor_ms": round(t_floor * 1e3, 4), "floor_parts": parts,
                       "peak_source": "algorithmic bytes / gather floor at the random-gather rates measured in this "
                                      "run (index-sized buffer: L2; 1.5 GiB: HBM, for the text checks)",
                       "index_gather_gbs": round(ceil["gbs"], 1), "hbm_gather_gbs": round(hbm["gbs"], 1)}
    return out


def run_uneven(args):
    import torch
    import paper_1402_4876_gb300 as mica
    dev = torch.device("cuda", 0)
    g = synth.genome_64m()
    idx = mica.Index.build(synth.to_acgt_bytes(g.codes), kmer_q=12, sa_sample=16)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    leg = uneven_leg(mica, idx, g, args.reads, args.steps, args.warmup, torch.cuda.current_stream(dev), flush,
                     headline=args.kernel)
    out = {"metric": "reads/s aligned, uneven batch (lengths 50/100/150/250, k 0-3)", "value": leg["value"],
           "unit": "reads/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
           "dtype": "u32", "data": "synthetic", "config": {"workload": leg["workload"]}, "uneven": leg}
    print(json.dumps(out), flush=True)


def human_leg(mica, dev, stream, pairs: int, genome_bp: int, steps: int = 2, plain: bool = True,
              batch: int = 2_000_000, pairing: bool = True, headline: str = "bidirectional") -> dict:
    """Human-scale: a synthetic genome of `genome_bp` (about 45% repeats) with
    its index resident in HBM, and `pairs` read pairs (2 x 150 bp mates, 0.1%
    donor variants + 1% sequencing error), each mate searched with k <= 2,
    cap 1000, in batches of `batch` mates.  Each batched kernel (the headline
    first) runs every batch `steps` times (the time is the mean), the plain
    kernel once; the index (3.3 GB) is larger than L2, so no flush is needed
    between steps."""
    import torch
    t0 = time.perf_counter()
    g = synth.human_genome(genome_bp)
    donor = synth.donor_of(g)
    b = synth.paired_reads(donor, pairs)
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    acgt = synth.to_acgt_bytes(g.codes)
    n_genome = g.n
    del g, donor
    idx = mica.Index.build(acgt, kmer_q=12, sa_sample=16)
    del acgt
    build_s = time.perf_counter() - t0
    info = idx.info()
    res = {}
    paired, pair_ms = 0, 0.0
    other = "persistent" if headline == "bidirectional" else "bidirectional"
    kernels = (headline, other) + (("plain",) if plain else ())
    for kernel in kernels:
        tot_ms, tot_kms, nodes, blocks, seeds, hits, ivs, retries = 0.0, 0.0, 0, 0, 0, 0, 0, 0
        vbytes, vsect, verified = 0, 0, 0
        reps = steps if kernel != "plain" else 1
        for r0 in range(0, b.n, batch):
            sub = b.subset(np.arange(r0, min(b.n, r0 + batch))) if b.n > batch else b
            d = _device_batch(sub, dev)
            # one untimed call on the batch first (a first call per shape may capture its launch sequence)
            ms, kms, st, r = _time_kernel(idx, d, sub.n, kernel, reps, 1, stream)
            if kernel == headline and pairing:
                # mate pairing of the batch's device result (outside the timed search)
                _, o, h = r.tensors()
                pout = torch.zeros(sub.n // 2 * mica.PAIR_DTYPE.itemsize, dtype=torch.uint8, device=dev)
                p0 = torch.cuda.Event(enable_timing=True)
                p1 = torch.cuda.Event(enable_timing=True)
                p0.record(stream)
                mica.pair_device(o, h, d[2], sub.n // 2, PAIR_WINDOW[0], PAIR_WINDOW[1], pout, stream=stream)
                p1.record(stream)
                p1.synchronize()
                pair_ms += p0.elapsed_time(p1)
                pr = pout.cpu().numpy().view(mica.PAIR_DTYPE)
                paired += int(np.count_nonzero(pr["n_concordant"]))
            tot_ms += statistics.mean(ms)
            tot_kms += statistics.mean(kms)
            nodes += st["nodes"]
            blocks += st["rank_blocks"]
            seeds += st["seeds"]
            ivs += st["intervals"]
            retries += st["retries"]
            vbytes += st["verify_bytes"]
            vsect += st["verify_sectors"]
            verified += st["verified"]
            hits += r.n_hits
        res[kernel] = {"value": round(b.n / (tot_ms / 1e3), 1), "pairs_per_s": round(b.n / 2 / (tot_ms / 1e3), 1),
                       "ms_total": round(tot_ms, 1), "kernel_ms_total": round(tot_kms, 1), "nodes": int(nodes),
                       "rank_blocks": int(blocks), "seeds": int(seeds), "intervals": int(ivs),
                       "verified": int(verified), "verify_bytes": int(vbytes), "verify_sectors": int(vsect),
                       "retries": int(retries), "hits": int(hits)}
    peaks, src = measured_peaks()
    p = res[headline]
    read_bytes = 4 * int(np.sum((b.lengths.astype(np.int64) + 15) // 16))
    alg = search_alg_bytes(headline, p, read_bytes)
    achieved = alg / (p["kernel_ms_total"] / 1e3) / 1e9
    hot = int(info["occ_bytes"] + info["rev_occ_bytes"] + info["table_bytes"] + info["rev_table_bytes"])
    ceil = mica.gather_ceiling((hot + 31) // 32 * 32, 32, loads=1 << 27, repeats=3)
    t_floor, floor_parts = gather_floor(headline, p, read_bytes, ceil["gbs"], ceil["gbs"], peaks["hbm_gbs"])
    peak = alg / t_floor / 1e9
    traffic = profile_traffic(BIDIR_CU if headline == "bidirectional" else SEARCH_CU,
                              PROFILE_BIDIR_HUMAN if headline == "bidirectional" else PROFILE_HUMAN,
                              "dram_bytes_search_step")
    n_batches = max(1, -(-b.n // batch))
    out = {"workload": f"{n_genome / 1e9:.2f} Gbp synthetic genome (~45% repeats), index resident in HBM; "
                       f"{pairs} pairs (2x150 bp), k<=2 per mate, cap 1000",
           "value": p["value"], "unit": "mates/s", "kernel": KERNEL_LABEL[headline],
           "batch_mates": min(batch, b.n), "steps": steps,
           "index_bytes": int(info["occ_bytes"] + info["mark_bytes"] + info["sample_bytes"] + info["table_bytes"]
                              + info["rev_occ_bytes"] + info["rev_table_bytes"]),
           headline: res[headline], other: res[other],
           f"{headline}_over_{other}": round(res[headline]["value"] / res[other]["value"], 3),
           "generate_s": round(gen_s, 1), "index_build_s": round(build_s, 1),
           "roofline": {"bound": "hbm_random_gather", "achieved": round(achieved, 1), "peak": round(peak, 1),
                        "unit": "GB/s", "frac": round(t_floor / (p["kernel_ms_total"] / 1e3), 4),
                        "traffic": traffic, "kernel": KERNEL_NAMES[headline],
                        "alg_bytes_per_launch": int(alg / n_batches), "alg_bytes_what": ALG_LABEL[headline],
                        "peak_source": f"the step's algorithmic bytes / its gather floor: the least time its "
                                       f"sectors take at the random 32 B gather rate measured in this run over "
                                       f"{hot >> 20} MiB (the index's occurrence blocks and q-mer tables of both "
                                       f"directions: HBM; the text-check arrays are HBM too), reads at the copy "
                                       f"bandwidth; frac = floor / kernel time",
                        "floor_ms": round(t_floor * 1e3, 3), "floor_parts": floor_parts,
                        "random_gather_gbs": round(ceil["gbs"], 1),
                        "frac_of_random_gather_by_bytes": round(achieved / ceil["gbs"], 4),
                        "hbm_copy_peak": peaks["hbm_gbs"], "frac_of_hbm_copy": round(achieved / peaks["hbm_gbs"], 4),
                        "hbm_copy_peak_source": f"{src} hbm_gbs (MEASURED_PEAKS.json)"}}
    if "plain" in res:
        out["plain"] = res["plain"]
        out["batched_over_plain"] = round(res[headline]["value"] / res["plain"]["value"], 3)
    if pairing:
        out["pairing"] = {"properly_paired": round(paired / (b.n // 2), 4), "window": list(PAIR_WINDOW),
                          "kernel_ms_total": round(pair_ms, 1),
                          "what": "pairs with a concordant placement (opposite strands, fragment in the window) "
                                  "among their listed hits; mica_pair_device after each batch"}
    idx.free()
    return out


def run_human(args):
    """Human-scale workload on its own: all `--pairs` pairs in batches of 2M mates."""
    import torch
    import paper_1402_4876_gb300 as mica
    dev = torch.device("cuda", 0)
    leg = human_leg(mica, dev, torch.cuda.current_stream(dev), args.pairs, args.genome_bp, steps=1,
                    headline=args.kernel)
    out = {"metric": "150bp mates/s aligned (k<=2 FM search), human-scale genome", "value": leg["value"],
           "unit": "reads/s", "n_gpus": 1, "higher_is_better": True, "dtype": "u32", "data": "synthetic",
           "config": {"workload": leg["workload"]}, "human": leg}
    print(json.dumps(out), flush=True)


def run_serve(args):
    """Serving: requests of log-uniform size (1e3..1e6 reads; lengths
    100/150/250, k 0..2) drawn from the human-scale donor arrive as a Poisson
    process at 50/70/90% of the sustained rate into the continuous-batching
    server over the resident 3.1 Gbp index; p50/p99 latency is submit to
    completion on the host clock.  Arrivals are open-loop: a submitting thread
    follows the drawn schedule, another thread collects results."""
    import threading
    import torch
    import paper_1402_4876_gb300 as mica
    g = synth.human_genome(args.genome_bp)
    donor = synth.donor_of(g)
    acgt = synth.to_acgt_bytes(g.codes)
    n_genome = g.n
    del g
    t0 = time.perf_counter()
    idx = mica.Index.build(acgt, kmer_q=12, sa_sample=16)
    build_s = time.perf_counter() - t0
    del acgt
    size_range = (1_000, args.serve_max_size)
    n_req = args.serve_requests
    workers, chunk, tick = 2, args.serve_chunk, args.serve_tick

    def run_level(reqs, gaps):
        lat, done = [None] * len(reqs), [0]
        with mica.Server(idx, hit_cap=HIT_CAP, workers=workers, chunk_reads=chunk, max_tick_reads=tick,
                         kernel=args.serve_kernel) as srv:
            ids = [None] * len(reqs)
            ready = threading.Semaphore(0)

            def submitter():
                t_next = time.perf_counter()
                for j, (gap, r) in enumerate(zip(gaps, reqs)):
                    t_next += gap
                    dt = t_next - time.perf_counter()
                    if dt > 0:
                        time.sleep(dt)
                    ids[j] = srv.submit_batch(r)
                    ready.release()

            th = threading.Thread(target=submitter)
            t_start = time.perf_counter()
            th.start()
            for j in range(len(reqs)):
                ready.acquire()
                _, lat[j] = srv.wait(ids[j])
            el = time.perf_counter() - t_start
            th.join()
            st = srv.stats()
        return lat, el, st

    # sustained rate: 16 requests queued back to back
    base = synth.serve_requests(donor, 16, seed=synth.SEED_READS_SERVE, size_range=size_range)
    _, el, st = run_level(base, [0.0] * len(base))
    sustained = sum(r.n for r in base) / el
    levels = {}
    clocks = []
    for li, frac in enumerate((0.5, 0.7, 0.9)):
        reqs = synth.serve_requests(donor, n_req, seed=synth.SEED_READS_SERVE + 1 + li, size_range=size_range)
        rng = np.random.default_rng(synth.SEED_ARRIVALS + li)
        mean_reads = np.mean([r.n for r in reqs])
        rate = frac * sustained / mean_reads                     # requests per second
        gaps = rng.exponential(1.0 / rate, size=len(reqs))
        with ClockSampler(0) as clk:
            lat, el, st = run_level(reqs, gaps)
        clocks.append(clk.summary())
        sizes = np.array([r.n for r in reqs])
        lat = np.array(lat)
        small = sizes <= np.percentile(sizes, 50)
        levels[f"{int(frac * 100)}%"] = {
            "p50_ms": round(float(np.percentile(lat, 50)), 2), "p99_ms": round(float(np.percentile(lat, 99)), 2),
            "p50_ms_smaller_half": round(float(np.percentile(lat[small], 50)), 2),
            "p99_ms_smaller_half": round(float(np.percentile(lat[small], 99)), 2),
            "offered_reads_per_s": round(frac * sustained, 1),
            "reads_per_s": round(int(sizes.sum()) / el, 1), "requests": len(reqs), "wall_s": round(el, 2),
            "ticks": int(st["ticks"]), "device_bytes_in_use": int(st["device_bytes_in_use"]),
            "clocks": clocks[-1]}
        del reqs
    out = {"metric": "serving: p50/p99 request latency and sustained reads/s", "value": round(sustained, 1),
           "unit": "reads/s", "n_gpus": 1, "higher_is_better": True, "dtype": "u32", "data": "synthetic",
           "config": {"workload": f"{n_genome / 1e9:.2f} Gbp genome resident; Poisson requests of log-uniform "
                                  f"{size_range[0]}..{size_range[1]} reads (100/150/250 bp, k 0..2)",
                      "workers": workers, "chunk_reads": chunk, "max_tick_reads": tick, "kernel": args.serve_kernel,
                      "requests_per_level": n_req,
                      "index_build_s": round(build_s, 1)},
           "levels": levels}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# the oracle on the host cores
# ---------------------------------------------------------------------------

def cpu_baseline(g, b, stride: int = 20):
    import oracle
    cores, model = cpu_info()
    fm = oracle.FMIndex(g.codes, "sais")                 # index build: not timed
    sub = b.subset(np.arange(0, b.n, stride))
    t = time.perf_counter()
    res = fm.align(sub, cap=HIT_CAP, threads=cores)
    dt = time.perf_counter() - t
    one = sub.subset(np.arange(0, sub.n, 8))             # an eighth of the sample on one core
    t = time.perf_counter()
    fm.align(one, cap=HIT_CAP, threads=1)
    dt1 = time.perf_counter() - t
    return {"value": round(sub.n / dt, 1), "unit": "reads/s", "cores": cores, "kind": "oracle",
            "sample": f"{sub.n} of the {b.n} reads (every {stride}th), same genome; oracle index build "
                      f"(SA-IS) excluded; {dt:.1f} s wall", "cpu": model,
            "one_core": {"value": round(one.n / dt1, 1), "unit": "reads/s",
                         "sample": f"every 8th read of that sample ({one.n} reads), {dt1:.1f} s wall"},
            "nodes_per_read": round(res.nodes / max(sub.n, 1), 1),   # plain backtracking, no table, no pruning
            }


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    import oracle
    cores, model = cpu_info()
    g, b = make_workload(args.reads, 0)
    fm = oracle.FMIndex(g.codes, "sais")
    stride = 50
    sub = b.subset(np.arange(0, b.n, stride))
    for _ in range(args.warmup):
        fm.align(sub.subset(np.arange(min(sub.n, 2000))), cap=HIT_CAP, threads=cores)
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        fm.align(sub, cap=HIT_CAP, threads=cores)
        times.append(time.perf_counter() - t)
    value = sub.n / statistics.mean(times)
    sample = (f"each step: {sub.n} of the {b.n} reads (every {stride}th); oracle index build excluded; "
              f"warm-up steps on 2,000 reads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": "reads/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * statistics.mean(times), 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic", "config": {"workload": WORKLOAD, "genome_bp": g.n, "reads": b.n, "hit_cap": HIT_CAP},
        "cpu_baseline": {"value": round(value, 1), "unit": "reads/s", "cores": cores, "kind": "oracle",
                         "sample": sample, "cpu": model},
        "e2e": {"value": round(value, 1), "unit": "reads/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "repeats64m":
        run_ours(args)
    elif args.workload == "uneven":
        run_uneven(args)
    elif args.workload == "human":
        run_human(args)
    else:
        run_serve(args)


if __name__ == "__main__":
    main()
