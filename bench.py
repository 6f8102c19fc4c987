"""Benchmark: batched enumeration of weak pseudo-manifolds on one GB300 (or N, weak scaling).

Workload (default): 4096 seeded Picard-4 instances, n uniform in {3..8}, dual maps with
m = n + 4 distinct nonzero rows of rank 4, property = the upper-bound-theorem cap; every
instance's full sorted list of WPM facet masks. One step = one batched run of the whole
path (candidate facets, ridges, search, per-instance sort) over the 4096 instances.

  value  search nodes/s of the whole job, outputs kept on the device, timed with CUDA
         events on the run's stream (inputs are host-side maps of 64 bytes each; the
         library copies their descriptors in the same step)
  e2e    the same metric through the C ABI with host buffers: the step includes copying
         the inputs in and every sorted mask list out to the caller's host arrays (through
         the library's page-locked staging buffer)

  plain_configs  the single-map workloads (Fano n = 3 and n = 5 maps, 16 seeds each, full
         lists; the whole n = 11 map, count only), one plain call per map
  paper_table1  every IDCM orbit of n = 8..11 under the cap alone (the paper's Table 1
         workload), seconds per orbit beside the paper's times (other hardware, other
         algorithm: context only)
  paper_table2  Algorithm 4.4 end to end for n = 2..10 (all four printed rows of Table 2),
         checked against the paper's counts, seconds per n
  paper_n11  Section 4.4's n = 11 construction end to end (114 links, then the paper's
         4 seeds), checked against the paper's counts, seconds
  paper_sweep  Section 2.1's GF(2) sweeps on the GPU: all 2^s kernel elements vs the convenient
         basis (Z blocks, fixed coordinates), combinations visited and seconds, on the Fano
         maps and Table 2's first row at n = 4, 5, 6
  paper_main_theorem  the main theorem's Picard-4 row assembled from the two runs above
         (plus Section 4.3's cross-polytope at n = 4): total against the paper's 3153
  serving  the request loop over the serving engine (continuous batching): Poisson
         arrivals at 200 jobs/s for 60 s, n uniform in {5..9}, each job's full sorted list;
         p50/p99 latency (completion - arrival) over the jobs finished by the deadline,
         throughput, and the jobs still queued or running then (N = 1 only)

--impl reference times the CPU oracle (the test oracle, unmodified) on a bounded sample of
the same workload. Under torchrun each rank runs its own seeded 4096-instance batch (weak
scaling, no collective on the data path); rank 0 prints the JSON line.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "search nodes/sec (batched, 4096 Picard-4 instances n=3..8)"
UNIT = "nodes/s"

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of the depth-first kernel per
# search node in list mode, from one ncu capture of the current kernel: one pass over 256 maps
# of this mix, 361,736,704 + 733,481,984 bytes for 2,711,713,518 nodes (masks written and work
# handed over included). None whenever the kernel has changed since its capture. The
# roofline's traffic scales it by the step's nodes.
TDFS_DRAM_BYTES_PER_NODE = (361736704 + 733481984) / 2711713518


# ------------------------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline): a spawn pool over sampled instances
# ------------------------------------------------------------------------------------------

def _oracle_job(args):
    k, kind, n, m, cols, keep = args
    import oracle as O
    f = O.candidate_facets(kind, n, m, cols)
    # room for every list of this workload (the oracle searches again when a list overflows)
    c, nodes, probes, masks = O.enumerate_dfs(n, m, f, cap=O.CAP_UBT, list_mode=True,
                                              capacity=1 << 20)
    return k, c, nodes, probes, (masks if keep else None)


def oracle_sample(insts, stride):
    """Every stride-th instance of the batch (a bounded, deterministic sample), with its
    index in the batch."""
    return [(k, i) for k, i in enumerate(insts) if k % stride == 0]


def time_oracle(sample, cores, keep=False):
    """The oracle over the sample in a spawn pool: (nodes, seconds, {index: (count, nodes,
    probes, sorted masks or None)})."""
    import oracle as O
    O.oracle.build()
    ctx = mp.get_context("spawn")
    # longest first (the search grows about 5x per unit of n), so the pool stays busy
    jobs = sorted(((k, i.kind, i.n, i.m, list(i.cols), keep) for k, i in sample),
                  key=lambda j: -j[2])
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = list(pool.imap_unordered(_oracle_job, jobs, chunksize=1))
    dt = time.perf_counter() - t0
    return sum(r[2] for r in res), dt, {r[0]: r[1:] for r in res}


def parity_sample(oracle_res, out, dev_out, words):
    """The timed run's last step against the oracle on the sampled maps: per map the count,
    node and probe counts, and the sorted mask list read back from the device buffers."""
    import numpy as np
    bad = []
    for k, (c, nodes, probes, masks) in sorted(oracle_res.items()):
        r = out[k]
        if (r.status, r.count, r.nodes, r.probes) != (0, c, nodes, probes):
            bad.append({"map": k, "gpu": [r.status, r.count, r.nodes, r.probes],
                        "oracle": [0, c, nodes, probes]})
            continue
        w = words[k]
        got = dev_out[k][: c * w].cpu().numpy().view(np.uint64).reshape(c, w)
        if not np.array_equal(got, masks):
            bad.append({"map": k, "masks_differ": True})
    return {"maps": len(oracle_res), "exact": not bad, "mismatches": bad[:8],
            "compared": "status, count, nodes, probes and the sorted mask list of each "
                        "sampled map (every stride-th of the batch), from the last timed step"}


# ------------------------------------------------------------------------------------------
# clocks
# ------------------------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int, path: str):
        self.path = path
        self.proc = None
        self.index = index

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}",
                                          f"--query-gpu={self.QUERY}", "--format=csv,noheader",
                                          "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        try:
            rows = [l.strip().split(", ") for l in open(self.path) if l.strip()]
        except Exception:
            rows = []
        mhz, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                mhz.append(float(r[1].split()[0]))
                mx = float(r[2].split()[0])
                for nm, v in zip(names, r[5:9]):
                    if v.strip() == "Active":
                        reasons.add(nm)
            except Exception:
                continue
        return {"sm_mhz": statistics.median(mhz) if mhz else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(mhz)}


# ------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------

def algorithmic_ops(res, insts):
    """Integer operations the canonical tree requires (the roofline's numerator): each tried
    child (node or probe) tests its n ridge counters (load, shift, test: 3 ops each), and each
    accepted child updates its n counters on entry and on exit (load, add, store: 6 ops)."""
    return sum(3 * i.n * (r.nodes + r.probes) + 6 * i.n * r.nodes for r, i in zip(res, insts))


def word_ops(res, insts):
    """The same work counted in 64-bit words: per node a select over ceil(N/64) words, per
    tried child its n counter tests, per accepted child n counter updates and ceil(M/64)
    words of Out."""
    tot = 0
    for r, i in zip(res, insts):
        wn, wm = (r.N + 63) // 64, (r.M + 63) // 64
        tot += r.nodes * wn + (r.nodes + r.probes) * i.n + r.nodes * (i.n + wm)
    return tot


def run_serving(args, rate=None, seconds=None, deadline=None):
    """The serving measurement: seeded Poisson arrivals served in real time by the engine."""
    from paper_2301_00806_gb300 import instances as I, serving
    rate = args.serve_rate if rate is None else rate
    seconds = args.serve_seconds if seconds is None else seconds
    deadline = args.serve_deadline if deadline is None else deadline
    jobs = I.poisson_jobs(rate=rate, duration=seconds, n_lo=5, n_hi=9, seed=args.seed)
    st = serving.serve(jobs, list_mode=True, max_n=9, deadline_s=deadline)
    sm = st.summary()
    done_nodes = st.nodes
    return {
        "workload": f"Poisson arrivals {rate:g}/s for {seconds:g} s, "
                    f"n~U{{5..9}}, m=n+4 dual maps, UBT cap, full sorted lists",
        "jobs": sm["jobs"], "completed": sm["completed"], "failed": sm["failed"],
        "unfinished_at_deadline": sm["jobs"] - sm["completed"] - sm["failed"],
        "deadline_s": deadline, "wall_s": sm["wall_s"],
        "p50_ms": sm["p50_ms"], "p99_ms": sm["p99_ms"], "mean_ms": sm["mean_ms"],
        "jobs_per_s": sm["jobs_per_s"], "nodes_per_s": sm["nodes_per_s"],
        "mean_nodes_per_completed_job": done_nodes / max(1, sm["completed"]),
        "engine_steps": sm["engine_steps"], "max_active_jobs": sm["max_active_jobs"],
        "latency": "completion minus arrival, over the jobs completed by the deadline",
    }


def run_serving_batched(args):
    """The serving workload's jobs (the sustained run's arrivals), all at once through one
    batched call: the nodes/s the same job mix reaches without arrivals, the reference the
    served throughput is compared with."""
    import torch
    from paper_2301_00806_gb300 import instances as I, wpm
    jobs = I.poisson_jobs(rate=args.serve_sustained_rate, duration=args.serve_sustained_seconds,
                          n_lo=5, n_hi=9, seed=args.seed)
    specs = [wpm.BatchSpec("dual", j.n, j.m, j.cols, cap=wpm.CAP_UBT) for j in jobs]
    counts = wpm.enumerate_batch(specs, list_mode=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = wpm.enumerate_batch(specs, list_mode=True, capacities=[max(1, r.count) for r in counts],
                              words=[r.words for r in counts])
    dt = time.perf_counter() - t0
    nodes = sum(r.nodes for r in res)
    return {"jobs": len(jobs), "nodes": nodes, "seconds": dt, "nodes_per_s": nodes / dt,
            "mode": "one wpm_enumerate_batch call, full sorted lists to host memory"}


# Table 1 of the paper: time per IDCM orbit of its kernel sweep under the upper-bound cap,
# on an Nvidia Quadro A5000 (n = 11: the authors' estimate, not a run).
PAPER_TABLE1_SECONDS_PER_ORBIT = {8: 15 * 60.0, 9: 2 * 3600.0, 10: 12 * 86400.0,
                                  11: 3 * 365 * 86400.0}


def run_plain_configs(stream):
    """The single-map workloads, each map by one plain wpm_enumerate call (full sorted list,
    except the n = 11 map: count only): the Fano map (n = 3) for 16 seeds, n = 5 dual maps
    for 16 seeds, and the whole n = 11 map (all 15 nonzero rows of Z2^4, seed 0)."""
    import torch
    from paper_2301_00806_gb300 import instances as I, wpm
    out = {}
    cases = [("fano_n3", [I.fano_primal(s) for s in range(16)], True),
             ("dual_n5", [I.single_dual(5, s) for s in range(16)], True),
             ("full_n11", [I.full_dual_n11(0)], False)]
    for name, insts, lists in cases:
        i0 = insts[0]
        wpm.enumerate(i0.kind, i0.n, i0.m, i0.cols, cap=wpm.CAP_UBT, list_mode=False)  # warm-up
        torch.cuda.synchronize()
        nodes = count = 0
        t0 = time.perf_counter()
        for i in insts:
            r = wpm.enumerate(i.kind, i.n, i.m, i.cols, cap=wpm.CAP_UBT, list_mode=lists,
                              capacity=1 << 16)
            nodes += r.nodes
            count += r.count
        dt = time.perf_counter() - t0
        out[name] = {"maps": len(insts), "wpms": count, "nodes": nodes, "seconds": dt,
                     "nodes_per_s": nodes / dt, "maps_per_s": len(insts) / dt,
                     "mode": "list" if lists else "count"}
    return out


TABLE2 = {  # Table 2 of the paper: |K(n,4)| at lines 7 and 13, |K°(n,4)| at lines 15 and 19
    2: (90, 22, 2, 1), 3: (1119, 578, 5, 4), 4: (20383, 13679, 49, 20),
    5: (79877, 47012, 256, 142), 6: (322837, 204714, 1791, 733), 7: (503624, 310217, 2194, 1190),
    8: (469445, 305280, 1401, 776), 9: (224854, 140933, 381, 243), 10: (99374, 57956, 56, 39)}


def run_paper_table2(stream):
    """Algorithm 4.4 end to end for n = 2..10 (seeds.colorable_seeds): one map per IDCM orbit
    with the base facet and the cap (GPU), the post-filters Pic(K) = 4 and seedness (GPU),
    one representative per isomorphism class and the PL-sphere test of Lemma 3.3 (host).
    Each n timed end to end."""
    import torch
    from paper_2301_00806_gb300 import seeds
    rows, total = [], 0.0
    for n in sorted(TABLE2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        run = seeds.colorable_seeds(n, stream=stream)
        dt = time.perf_counter() - t0
        total += dt
        got = (run.line7, run.line13, run.line15, run.line19)
        rows.append({"n": n, "lines_7_13_15_19": list(got), "paper": list(TABLE2[n]),
                     "exact": got == TABLE2[n], "seconds": dt})
    return {"workload": "Algorithm 4.4 for n = 2..10: one map per IDCM orbit, base facet and "
                        "cap, post-filters (GPU), isomorphism classes and PL spheres (host)",
            "all_exact": all(r["exact"] for r in rows), "seconds_total": total, "rows": rows}


def run_paper_n11(stream):
    """Section 4.4's n = 11 construction end to end (seeds.colorable_seeds_n11): the n = 10
    run without the seedness discard gives the links (the paper: 114 PL spheres, 39 of them
    seeds); one conditioned n = 11 search per link, then Algorithm 4.4's filters (the paper's
    Theorem: exactly 4 seeds)."""
    import torch
    from paper_2301_00806_gb300 import seeds
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    links, run = seeds.colorable_seeds_n11(stream=stream)
    dt = time.perf_counter() - t0
    return {"workload": "n = 10 links (3 IDCM orbits, base facet and cap, Pic(K) = 4, "
                        "classes, PL spheres), then one cone-conditioned n = 11 search per link "
                        "with the cap, post-filters, classes and PL spheres",
            "links": links.line19, "n11_wpms": run.line7, "n11_pic_seed": run.line13,
            "n11_classes": run.line15, "n11_seeds": run.line19,
            "paper": {"links": 114, "n11_seeds": 4},
            "exact": links.line19 == 114 and run.line19 == 4,
            "nodes": links.nodes + run.nodes, "seconds": dt,
            "seconds_links": links.seconds, "seconds_n11": run.seconds}


def run_main_theorem(table2, n11, stream):
    """The main theorem's Picard-4 row from the two runs above: Table 2's line 19 per n,
    Section 4.3's cross-polytope at n = 4 (checked: a PL sphere isomorphic to none of the
    n = 4 classes), the n = 11 seeds; its total against the paper's 3153."""
    from paper_2301_00806_gb300 import seeds
    row = {r["n"]: r["lines_7_13_15_19"][3] for r in table2["rows"]}
    extra = seeds.extra_n4_seed(seeds.colorable_seeds(4, stream=stream))
    row[4] += int(extra)
    row[11] = n11["n11_seeds"]
    want = seeds.MAIN_THEOREM_P4
    return {"row": {str(k): v for k, v in sorted(row.items())}, "total": sum(row.values()),
            "paper_total": sum(want.values()), "cross_polytope_added": extra,
            "exact": row == want}


def _guarded(fn, *args):
    """An extra section's result, or its error (the main line is printed either way)."""
    try:
        return fn(*args)
    except Exception as e:  # noqa: BLE001
        return {"error": f"{type(e).__name__}: {e}"}


def run_paper_table1(stream):
    """Every IDCM orbit of n = 8..11 (one map each, the cap only, counting mode) as one
    batched run per n: seconds per orbit beside the paper's."""
    import torch
    from paper_2301_00806_gb300 import instances as I, wpm
    rows = []
    for n in sorted(PAPER_TABLE1_SECONDS_PER_ORBIT):
        reps = I.idcm_orbit_reps(n)
        specs = [wpm.BatchSpec("dual", n, n + 4, r, cap=wpm.CAP_UBT) for r in reps]
        wpm.enumerate_batch(specs[:1], list_mode=False, stream=stream)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = wpm.enumerate_batch(specs, list_mode=False, stream=stream)
        dt = time.perf_counter() - t0
        assert all(r.status == 0 for r in res)
        per = dt / len(reps)
        paper = PAPER_TABLE1_SECONDS_PER_ORBIT[n]
        rows.append({"n": n, "orbits": len(reps), "wpms": sum(r.count for r in res),
                     "nodes": sum(r.nodes for r in res), "seconds_per_orbit": per,
                     "paper_seconds_per_orbit": paper, "paper_over_ours": paper / per})
    return {"workload": "one map per IDCM orbit (Section 4.2), UBT cap only, counting mode, "
                        "each n one batched call timed end to end on the host",
            "paper_hardware": "Nvidia Quadro A5000, kernel-combination sweep (Algorithm 2.2); "
                              "n = 11 is the paper's estimate",
            "rows": rows}


def run_paper_sweep(stream):
    """The GF(2) sweeps of Section 2.1 on the GPU: the plain sweep of all 2^s kernel elements
    (engine 2) against the sweep over the convenient basis (engine 1: fixed coordinates, Z
    blocks), on the Fano maps and on Table 2's first row at n = 4, 5 and 6 (one map per IDCM
    orbit, base facet and cap); combinations visited, seconds, and the WPM totals, which must
    equal the paper's (and the search's)."""
    import torch
    from paper_2301_00806_gb300 import instances as I, wpm
    cases = [("fano_n3", [wpm.BatchSpec(i.kind, i.n, i.m, i.cols, cap=wpm.CAP_UBT)
                          for i in (I.fano_primal(s) for s in range(16))], 16 * 666),
             ("table2_n4", [wpm.BatchSpec("dual", 4, 8, r, cap=wpm.CAP_UBT, base_facet=True)
                            for r in I.idcm_orbit_reps(4)], TABLE2[4][0]),
             ("table2_n5", [wpm.BatchSpec("dual", 5, 9, r, cap=wpm.CAP_UBT, base_facet=True)
                            for r in I.idcm_orbit_reps(5)], TABLE2[5][0]),
             ("table2_n6", [wpm.BatchSpec("dual", 6, 10, r, cap=wpm.CAP_UBT, base_facet=True)
                            for r in I.idcm_orbit_reps(6)], TABLE2[6][0])]
    rows = []
    for name, specs, want in cases:
        row = {"case": name, "maps": len(specs), "paper_or_expected": want}
        for label, tun in (("plain", {"engine": 2}), ("blocks", {"engine": 1}),
                           ("search", {})):
            wpm.enumerate_batch(specs[:1], list_mode=False, tuning=tun or None, stream=stream)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = wpm.enumerate_batch(specs, list_mode=False, tuning=tun or None, stream=stream)
            dt = time.perf_counter() - t0
            row[label] = {"wpms": sum(r.count for r in res), "visited": sum(r.nodes for r in res),
                          "seconds": dt}
        row["exact"] = row["plain"]["wpms"] == row["blocks"]["wpms"] == row["search"]["wpms"] == want
        row["blocks_over_plain_visited"] = row["blocks"]["visited"] / row["plain"]["visited"]
        rows.append(row)
    return {"workload": "Section 2.1 sweeps: all 2^s elements of ker A (engine 2) vs the "
                        "convenient basis (engine 1); 'visited' = combinations (sweeps) or "
                        "search nodes (search)", "all_exact": all(r["exact"] for r in rows),
            "rows": rows}


def reduce_over_ranks(ms, nodes, launches, world, device):
    """Whole-job figures of a weak-scaling run: the slowest rank's time (max) and the nodes
    and launches of all ranks (sum). One rank: the inputs."""
    if world <= 1:
        return float(ms), float(nodes), float(launches)
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms, nodes, launches], dtype=torch.float64, device=device)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm = t.clone()
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(sm[1]), float(sm[2])


def run_ours(args, rank, world, oracle_res=None):
    import numpy as np
    import torch
    from paper_2301_00806_gb300 import instances as I, wpm

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", dev))

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    insts = I.batch_duals(args.count, 3, 8, seed=args.seed + rank)
    specs = [wpm.BatchSpec("dual", i.n, i.m, i.cols, cap=wpm.CAP_UBT) for i in insts]
    stream = torch.cuda.Stream()
    # the library's autotuner picks the search mode, frontier and hand-over chunk on a
    # sample of this batch (untimed); the timed steps run with its choice
    tuned, tune_ms = wpm.autotune(specs, stream=stream)
    tuning = {k: v for k, v in tuned.items() if v}
    tuning["profile"] = 1
    if args.pass_loop == "host":  # each depth-first pass launched by the host (profilers
        tuning["graph"] = -1      # cannot see kernels inside conditional graph nodes)

    # counts first (untimed): they size the output lists
    res = wpm.enumerate_batch(specs, list_mode=False, tuning=tuning, stream=stream)
    caps = [max(1, r.count) for r in res]
    words = [r.words for r in res]
    offs = np.concatenate([[0], np.cumsum([c * w for c, w in zip(caps, words)])])
    dev_buf = torch.empty(int(offs[-1]), dtype=torch.int64, device="cuda")
    dev_out = [dev_buf[int(offs[k]):int(offs[k + 1])] for k in range(len(specs))]
    nodes_step = sum(r.nodes for r in res)
    ops_step = algorithmic_ops(res, insts)
    ops_step_words = word_ops(res, insts)
    # the roofline's peak: integer instructions per second of this GPU, measured (untimed)
    peak_ops, _ = wpm.int_peak(0)
    peak_popc, _ = wpm.int_peak(1)

    def step_device():
        return wpm.enumerate_batch(specs, list_mode=True, capacities=caps, tuning=tuning,
                                   stream=stream, device_out=dev_out)

    for _ in range(args.warmup):
        step_device()
    torch.cuda.synchronize()
    clock = ClockSampler(dev, os.path.join(args.out_dir, f"clocks_rank{rank}.csv"))
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    dfs_ms = 0.0
    dfs_launches = 0
    launches = 0
    with clock:
        barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            out = step_device()
            st = wpm.last_run_stats()
            dfs_ms += st["dfs_ms"]
            dfs_launches += st["dfs_passes"]
            launches += st["kernel_launches"]
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
    ms = ev0.elapsed_time(ev1)
    assert all(r.status == 0 for r in out)
    assert sum(r.nodes for r in out) == nodes_step
    parity = parity_sample(oracle_res, out, dev_out, words) if oracle_res else None

    # end to end through the C ABI with host buffers (inputs in, sorted lists out), the
    # host output arrays allocated once and reused from step to step
    host_caps = caps
    host_out = [np.empty(max(c, 1) * w, dtype=np.uint64) for c, w in zip(caps, words)]
    e2e_times, e2e_parts, h2d, d2h = [], [], 0, 0
    for k in range(max(1, args.e2e_steps) + 1):  # the first call touches the host pages
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out_h = wpm.enumerate_batch(specs, list_mode=True, capacities=host_caps, tuning=None,
                                    stream=stream, words=words,
                                    host_out=host_out)  # NULL: the tuned choice
        if k == 0:
            e2e_first = time.perf_counter() - t0
            continue
        e2e_times.append(time.perf_counter() - t0)
        st = wpm.last_run_stats()
        h2d, d2h = st["h2d_bytes"], st["d2h_bytes"]
        e2e_parts.append((st["run_ms"], st["copy_out_ms"], st["host_copy_ms"]))
    assert sum(r.nodes for r in out_h) == nodes_step

    # the plain path: one instance per call, on a sample of the same batch
    plain = None
    if args.plain_sample > 0:
        stride = max(1, len(insts) // args.plain_sample)
        smp = [(s, i) for k, (s, i) in enumerate(zip(specs, insts)) if k % stride == 0]
        pn = 0
        t0 = time.perf_counter()
        for s, i in smp:
            r = wpm.enumerate(s.kind, s.n, s.m, s.cols, cap=s.cap, list_mode=False)
            pn += r.nodes
        pdt = time.perf_counter() - t0
        plain = {"value": pn / pdt, "unit": UNIT, "instances": len(smp),
                 "instances_per_s": len(smp) / pdt, "mode": "one wpm_enumerate call per instance"}

    ms_all, nodes_all, _ = reduce_over_ranks(ms, nodes_step * args.steps, launches, world,
                                             "cuda")
    if rank != 0:
        return None
    clocks = clock.summary()
    sec = ms_all / 1000.0
    value = nodes_all / sec
    inst_per_s = world * len(insts) * args.steps / sec
    e2e_t = statistics.median(e2e_times)
    from paper_2301_00806_gb300 import instances as _I  # noqa: F401
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    nominal_ops = n_sm * 128 * 2070.0 * 1e6
    achieved = ops_step * args.steps / (dfs_ms / 1000.0) if dfs_ms > 0 else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_all / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic (seeded dual maps; no dataset)",
        "config": {"workload": f"{args.count} Picard-4 dual maps, n~U{{3..8}}, m=n+4, UBT cap, "
                               f"full sorted WPM lists", "instances_per_gpu": args.count,
                   "seed": args.seed, "mode": "list", "parallelism": f"replicas x{world}",
                   "l2": "not flushed: each step streams GBs (work ring, output lists) through "
                         "the 129 MB L2",
                   "tuning": {k: v for k, v in tuning.items() if k != "profile"},
                   "pass_loop": args.pass_loop,
                   "tuning_from": "wpm_autotune on every 16th map of the batch"},
        "instances_per_s": inst_per_s,
        "nodes_per_step": nodes_step * world,
        "e2e": {"value": world * nodes_step / e2e_t, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_t * 1000.0,
                "ms_per_call": [round(t * 1000.0, 1) for t in e2e_times],
                "first_call_ms": round(e2e_first * 1000.0, 1),
                "library_ms_per_call": [round(p[0], 1) for p in e2e_parts],
                "copy_out_ms_per_call": [round(p[1], 1) for p in e2e_parts],
                "host_copy_ms_per_call": [round(p[2], 1) for p in e2e_parts]},
        "plain_launch": plain,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_ops, "unit": "int ops/s",
                     "frac": (achieved / peak_ops) if achieved else None,
                     "traffic": (TDFS_DRAM_BYTES_PER_NODE * nodes_step
                                 if TDFS_DRAM_BYTES_PER_NODE else None),
                     "traffic_per": "step (its depth-first launches), scaled from an ncu "
                                    "capture of the kernel in list mode by search nodes",
                     "kernel": "depth-first pass (tdfs_kernel)",
                     "dfs_launches_per_step": dfs_launches / args.steps,
                     "dfs_ms_per_step": dfs_ms / args.steps,
                     "ops_model": "3n per tried child + 6n per accepted child (n ridge counters "
                                  "tested, then updated on entry and exit); frac uses this",
                     "ops_per_node": ops_step / nodes_step,
                     "ops_per_node_word_count": ops_step_words / nodes_step,
                     "frac_word_count": (ops_step_words * args.steps / (dfs_ms / 1000.0) /
                                         peak_ops) if dfs_ms > 0 else None,
                     "peak_from": "measured: wpm_int_peak, independent lop3 + add chains on "
                                  "every SM (popc + xor chains: %.3g ops/s; nominal 152 x 128 "
                                  "x 2070 MHz: %.3g)" % (peak_popc, nominal_ops)},
        "gpu_launches": launches,
        "clocks": clocks,
        "parity_sample": parity,
    }
    if world == 1 and args.table1:
        line["plain_configs"] = run_plain_configs(stream)
        line["paper_table1"] = run_paper_table1(stream)
        line["paper_table2"] = _guarded(run_paper_table2, stream)
        line["paper_sweep"] = _guarded(run_paper_sweep, stream)
        line["paper_n11"] = _guarded(run_paper_n11, stream)
        if "rows" in line["paper_table2"] and "n11_seeds" in line["paper_n11"]:
            line["paper_main_theorem"] = _guarded(run_main_theorem, line["paper_table2"],
                                                  line["paper_n11"], stream)
    if world == 1 and args.serve_seconds > 0:
        line["serving"] = run_serving(args)
    if world == 1 and args.serve_sustained_seconds > 0:
        # a rate the GPU sustains: latency is then service time, not queueing
        line["serving_sustained"] = run_serving(args, rate=args.serve_sustained_rate,
                                                seconds=args.serve_sustained_seconds,
                                                deadline=2 * args.serve_sustained_seconds + 30)
        line["serving_batched_reference"] = _guarded(run_serving_batched, args)
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--count", type=int, default=4096)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--plain-sample", type=int, default=256)
    ap.add_argument("--cpu-stride", type=int, default=64, help="oracle sample: every k-th instance")
    ap.add_argument("--pass-loop", default="graph", choices=["graph", "host"],
                    help="depth-first passes as one CUDA graph launch, or launched by the host")
    ap.add_argument("--table1", type=int, default=1,
                    help="time every IDCM orbit of n = 8..11 beside the paper's Table 1")
    ap.add_argument("--serve-rate", type=float, default=200.0, help="serving: arrivals per s")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="serving: seconds of arrivals (0 = no serving run)")
    ap.add_argument("--serve-deadline", type=float, default=90.0,
                    help="serving: seconds after which the loop stops")
    ap.add_argument("--serve-sustained-rate", type=float, default=60.0,
                    help="serving at a rate the GPU sustains: arrivals per s")
    ap.add_argument("--serve-sustained-seconds", type=float, default=30.0,
                    help="seconds of arrivals at the sustained rate (0 = no such run)")
    ap.add_argument("--out-dir", default=os.path.join(ROOT, "bench_out"),
                    help="where the sampled clock log is written")
    args = ap.parse_args()
    os.makedirs(args.out_dir, exist_ok=True)
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()

    from paper_2301_00806_gb300 import instances as I
    if args.impl == "reference":
        if rank != 0:
            return
        insts = I.batch_duals(args.count, 3, 8, seed=args.seed)
        sample = oracle_sample(insts, args.cpu_stride)
        per_step = []
        total_nodes = 0
        for _ in range(args.warmup):
            time_oracle(sample[:2], cores)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            nodes, dt, _ = time_oracle(sample, cores)
            per_step.append(dt)
            total_nodes += nodes
        wall = time.perf_counter() - t0
        value = total_nodes / wall
        desc = f"every {args.cpu_stride}th of the {args.count} instances ({len(sample)} maps)"
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8/int",
            "data": "synthetic (seeded dual maps)",
            "config": {"workload": f"{args.count} Picard-4 dual maps, n~U{{3..8}}, UBT cap "
                                   f"(oracle on a sample)", "seed": args.seed},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
        }), flush=True)
        return

    # CPU baseline first (spawn pool, before any CUDA call), rank 0 at N=1 only
    cpu = None
    oracle_res = None
    if rank == 0 and world == 1 and args.cpu_stride > 0:
        insts = I.batch_duals(args.count, 3, 8, seed=args.seed)
        sample = oracle_sample(insts, args.cpu_stride)
        nodes, dt, oracle_res = time_oracle(sample, cores, keep=True)
        cpu = {"value": nodes / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"every {args.cpu_stride}th of the {args.count} instances "
                         f"({len(sample)} maps, {nodes} nodes, {dt:.1f} s)"}
    line = run_ours(args, rank, world, oracle_res)
    if line is not None:
        line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
        if line.get("parity_sample") and not line["parity_sample"]["exact"]:
            sys.exit("parity_sample: the GPU run differs from the oracle on sampled maps")
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
