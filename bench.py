"""CompaSO hot-path benchmark (one JSON line on rank 0).

A step is one pass of the whole hot path — kernel density, L0 FoF, L1 and L2
competitive SO, labels and catalogue — over one synthetic box.  The default
workload is the medium box: side 256 l_mean, 256^3 = 16.8M particles, 40%
uniform background and 60% in NFW haloes of 20-2e5 particles with 10%
satellites (seeded), int32 positions on a 2^21 grid.

  value  particles/s with the inputs resident in device memory
  e2e    particles/s through the same C-ABI call with pinned host buffers
         (host->device copy of positions and ids, device->host copy of the
         four per-particle outputs and the catalogue, inside the timed region)

--impl reference times the CPU oracle (single thread) on bounded samples of
the same recipe instead.  Under torchrun each rank runs its own box (weak
scaling, no collective on the data path).
"""
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

WORKLOADS = {
    "medium": dict(desc="medium box: side 256 l_mean, 16,777,216 particles, 40% background, 60% NFW haloes "
                        "N in [20, 2e5] (slope -1.9, c in [4, 12]), 10% with satellites"),
    "medium128": dict(desc="the medium recipe in a side-128 box: 2,097,152 particles (profiling size)"),
    "tiny": dict(desc="tiny box: side 64 l_mean, 262,144 particles, 50% background, 50% NFW haloes N in "
                      "[20, 2e4]"),
    "batched": dict(desc="pre-formed groups: 4,000,000 particles in a side-256 box, group sizes with equal "
                         "particles per log interval on [35, 2e6] plus one forced 2e6 giant, each an NFW host with "
                         "0-5 NFW subhaloes (mass ratio 0.01-0.3), groups isolated (no background)"),
    "batched_many": dict(desc="100,000 pre-formed groups of 35-45 particles (single NFW haloes), ~4.0M particles "
                              "in a side-256 box"),
}
OPS_PER_PAIR = 11  # 3 sub, 3 mul, 2 add for d; compare; b2 - d; accumulate
# DRAM bytes (read + write) of one k_density launch per workload, from the
# single-pass ncu capture summarised in profiles/ (only for the kernel as it
# stands; absent workloads report null)
DENSITY_DRAM_BYTES = {"medium": 3.2425e9}


def cell_table_bytes(u):
    """Bytes of the dense cell table of a whole box of spacing u (cells of
    side >= b = 0.4 u, uint32 offsets)."""
    import math
    b2 = round((0.4 * u) ** 2)
    nc = int((1 << 21) / math.sqrt(b2))
    while (1 << 42) < b2 * nc * nc:
        nc -= 1
    return 4 * (nc ** 3 + 1)


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,timestamp")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.p = None
        self.window = None  # (t0, t1) wall-clock seconds of the timed region

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            time.sleep(0.5)  # the sampler is running before the timed region opens
        except Exception:
            self.p = None
        return self

    def mark(self, which):
        """Record the wall clock at the start (0) or end (1) of the timed region."""
        if self.window is None:
            self.window = [None, None]
        self.window[which] = time.time()

    def __exit__(self, *a):
        self.out = ""
        if self.p:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        import datetime
        rows = []
        for line in (getattr(self, "out", "") or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(f[9], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append(dict(sm=float(f[1]), smax=float(f[2]), hw=f[5], hwt=f[6], swt=f[7], pcap=f[8], t=ts))
            except ValueError:
                continue
        if self.window and None not in self.window and rows:
            t0, t1 = self.window
            inside = [r for r in rows if t0 <= r["t"] <= t1]
            # a region shorter than the sampling period keeps the sample nearest its middle
            rows = inside or [min(rows, key=lambda r: abs(r["t"] - 0.5 * (t0 + t1)))]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        reasons = set()
        for r in rows:
            for k, nm in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"), ("swt", "sw_thermal_slowdown"),
                          ("pcap", "sw_power_cap")):
                if r[k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(r["sm"] for r in rows), "sm_max_mhz": max(r["smax"] for r in rows),
                "samples": len(rows), "reasons": sorted(reasons)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def whole_job_rate(n_per_rank, ms_local, world_size, dist=None, device="cpu"):
    """Whole-job throughput of a weak-scaling run: every rank processes its
    own box of n_per_rank particles; the job takes as long as the slowest
    rank.  Returns (particles/s over all ranks, max ms over ranks)."""
    ms = float(ms_local)
    if dist is not None and world_size > 1:
        import torch
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return world_size * n_per_rank / (ms / 1e3), ms


def make_workload_seed(rank, base=20211022):
    """Seed of the medium box of one rank (every rank draws its own box)."""
    return base + 1000 * rank


def make_workload(name, seed_offset):
    from paper_2110_11408_gb300 import synth
    if name == "medium":
        return synth.medium(seed=make_workload_seed(seed_offset, synth.SEED0 + 1))
    if name == "tiny":
        return synth.tiny(seed=synth.SEED0 + 1000 * seed_offset)
    if name == "medium128":
        return synth.medium_sample(side=128, seed=synth.SEED0 + 11 + 1000 * seed_offset)
    if name == "batched":
        return synth.batched(seed=synth.SEED0 + 3 + 1000 * seed_offset)
    if name == "batched_many":
        return synth.batched_many(seed=synth.SEED0 + 4 + 1000 * seed_offset)
    raise SystemExit("unknown workload " + name)


def served_stream(cso, torch, local, flags, n_req=24, n_distinct=6, mean_gap_s=0.020, seed=7):
    """Poisson arrivals of boxes of the medium recipe at side 128 (2,097,152
    particles each, the size of one 1/64 slab of a side-512 box) submitted to
    the served path; latency = completion - scheduled arrival."""
    from paper_2110_11408_gb300 import synth
    rng = np.random.default_rng(seed)
    data = [synth.medium_sample(side=128, seed=synth.SEED0 + 300 + k) for k in range(n_distinct)]
    dev = [(torch.from_numpy(p).cuda(), torch.from_numpy(i.view(np.int64)).cuda(), m) for p, i, m in data]
    gaps = rng.exponential(mean_gap_s, n_req)
    out = {}
    for label, arrivals in (("poisson", np.cumsum(gaps)), ("saturated", np.zeros(n_req))):
        ctx = cso.Context(local, flags=flags | cso.FLAG_SLOTS(4))
        # warm the slots (workspace growth happens once per slot)
        warm = [cso.Buffers(dev[k % n_distinct][0], dev[k % n_distinct][1], True) for k in range(4)]
        wt = [ctx.submit(b, cso.cso_params_default(dev[0][2]["u"])) for b in warm]
        for t in wt:
            ctx.wait(t)
        bufs, tickets, sched = [], [], []
        t0 = cso.cso_clock() + 0.01
        for k in range(n_req):
            pos, ids, meta = dev[k % n_distinct]
            b = cso.Buffers(pos, ids, True)
            target = t0 + arrivals[k]
            while cso.cso_clock() < target:
                pass
            bufs.append(b)
            sched.append(target)
            tickets.append(ctx.submit(b, cso.cso_params_default(meta["u"])))
        for t in tickets:
            done, rc = ctx.wait(t)
            assert done and rc == 0, cso.cso_last_error()
        done_t = np.array([cso.cso_ticket_times(ctx.h, t)[2] for t in tickets])
        lat = (done_t - np.array(sched)) * 1e3
        n_tot = sum(len(dev[k % n_distinct][0]) for k in range(n_req))
        span = done_t.max() - min(sched)
        out[label] = {"requests": n_req, "particles_per_request": int(len(dev[0][0])), "slots": 4,
                      "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                      "particles_per_s": n_tot / span,
                      "arrivals": ("Poisson, mean gap %.0f ms" % (mean_gap_s * 1e3)) if label == "poisson"
                      else "all at t = 0"}
        ctx.close()
    return out


def slab_stream(cso, torch, local, flags, pos, ids, meta, n_slabs=64, mean_gap_s=0.020, seed=11):
    """The benchmark box delivered as n_slabs x-slabs in order (ghost columns
    and open L0 groups stay on the device between slabs).  Latency = the time
    from a slab's scheduled arrival until all its particles have final labels;
    the first slabs wait for the periodic seam, which closes with the last."""
    box = 1 << 21
    rng = np.random.default_rng(seed)
    edges = [box * k // n_slabs for k in range(n_slabs + 1)]
    order = np.argsort(pos[:, 0], kind="stable")
    xs = pos[order, 0]
    cuts = np.searchsorted(xs, edges)
    slabs = []
    for k in range(n_slabs):
        sl = order[cuts[k]:cuts[k + 1]]
        slabs.append((torch.from_numpy(np.ascontiguousarray(pos[sl])).cuda(),
                      torch.from_numpy(np.ascontiguousarray(ids[sl]).view(np.int64)).cuda()))
    params = cso.cso_params_default(meta["u"])
    out = {}
    for label, gaps in (("poisson", rng.exponential(mean_gap_s, n_slabs)), ("saturated", np.zeros(n_slabs))):
        arrivals = np.cumsum(gaps) if label == "poisson" else gaps
        ctx = cso.Context(local, flags=flags | cso.FLAG_SLOTS(2))
        bufs, tickets, sched = [], [], []
        t0 = cso.cso_clock() + 0.01
        for k in range(n_slabs):
            sp, si = slabs[k]
            b = cso.Buffers(sp, si, True, halo_cap=len(sp) // 20 + 64, x_lo=edges[k], x_hi=edges[k + 1],
                            request_id=1000 + k // n_slabs + (0 if label == "poisson" else 1))
            target = t0 + arrivals[k]
            while cso.cso_clock() < target:
                pass
            bufs.append(b)
            sched.append(target)
            tickets.append(ctx.submit(b, params))
        for t in tickets:
            done, rc = ctx.wait(t)
            assert done and rc == 0, cso.cso_last_error()
        done_t = np.array([cso.cso_ticket_times(ctx.h, t)[2] for t in tickets])
        lat = (done_t - np.array(sched)) * 1e3
        span = done_t.max() - min(sched)
        out[label] = {"slabs": n_slabs, "particles": int(len(pos)), "p50_ms": float(np.percentile(lat, 50)),
                      "p99_ms": float(np.percentile(lat, 99)), "particles_per_s": len(pos) / span,
                      "arrivals": ("Poisson, mean gap %.0f ms" % (mean_gap_s * 1e3)) if label == "poisson"
                      else "all at t = 0"}
        ctx.close()
    return out


SERVED_SCALE = {
    "served512": dict(box="served512", budget_gb=40, small=(), desc=(
        "served stream: periodic box side 512 l_mean, 134,217,728 particles (40% background, 60% NFW haloes N in "
        "[20, 2e6], 10% with satellites), delivered as 64 x-slabs of 8 l_mean (~2.1M particles) with Poisson "
        "arrivals (mean gap 20 ms) under a 40 GB device budget")),
    "served1024": dict(box="served1024", budget_gb=120, small=(64, 128, 256), desc=(
        "served stream at scale: periodic box side 1024 l_mean, 1,073,741,824 particles (same mixture, N up to "
        "1e7), delivered as 256 x-slabs of 1-4 columns of 2 l_mean with Poisson arrivals (mean gap 20 ms), "
        "interleaved with independent boxes of side 64/128/256 (262k-16.8M particles), under a 120 GB budget")),
}


def served_at_scale(args, cso, torch, local, name, emit=True):
    """A box streamed as x-slabs through the served path (cso_submit /
    cso_poll): slabs are generated untimed and kept in device memory, then
    submitted in x order at their scheduled arrival times; latency =
    completion - scheduled arrival.  Three passes over the same slabs: a
    warm-up (workspaces grow), Poisson arrivals, and all slabs at once (the
    throughput).  For the side-512 box the same particles also run as one
    whole box (plain and batched schedules), and the stream's labels are
    compared with the whole box's bit for bit."""
    from paper_2110_11408_gb300 import synth
    spec = SERVED_SCALE[name]
    box = getattr(synth, spec["box"])()
    workers = max(1, min(16, os.cpu_count() or 1))
    t0 = time.perf_counter()
    slabs = []
    for k, pos, ids in box.slabs(workers=workers, shuffle_seed=box.seed + 99):
        slabs.append((torch.from_numpy(pos).cuda(), torch.from_numpy(ids.view(np.int64)).cuda(),
                      int(box.edges[k]), int(box.edges[k + 1])))
    gen_s = time.perf_counter() - t0
    small = []
    for j, side in enumerate(spec["small"]):
        pos, ids, meta = synth.medium_sample(side=side, seed=synth.SEED0 + 700 + j)
        small.append((torch.from_numpy(pos).cuda(), torch.from_numpy(ids.view(np.int64)).cuda(), meta["u"]))
    torch.cuda.synchronize()
    n = sum(len(s[0]) for s in slabs)
    params = cso.cso_params_default(box.u)
    flags = cso.FLAG_BATCHED | cso.FLAG_SLOTS(4)
    budget = spec["budget_gb"] << 30
    rng = np.random.default_rng(box.seed + 7)

    def one_pass(label, gaps, request_id):
        ctx = cso.Context(local, budget_bytes=budget, flags=flags)
        arrivals = np.cumsum(gaps) if gaps is not None else np.zeros(len(slabs))
        n_small = 4 * len(small)
        small_at = np.sort(rng.uniform(0, arrivals[-1] if gaps is not None else 0.0, n_small)) if small else []
        bufs, tickets, sched, kinds = [], [], [], []
        torch.cuda.synchronize()
        t_base = cso.cso_clock() + 0.01
        si = 0
        for k, (pos, ids, x_lo, x_hi) in enumerate(slabs):
            while si < len(small_at) and small_at[si] <= arrivals[k]:
                sp, sd, su = small[si % len(small)]
                target = t_base + small_at[si]
                while cso.cso_clock() < target:
                    pass
                b = cso.Buffers(sp, sd, True, want=("l0", "l1", "l2"))
                bufs.append(b)
                sched.append(target)
                kinds.append(-1)
                tickets.append(ctx.submit(b, cso.cso_params_default(su)))
                si += 1
            target = t_base + arrivals[k]
            while cso.cso_clock() < target:
                pass
            b = cso.Buffers(pos, ids, True, halo_cap=len(pos) // 20 + 64, x_lo=x_lo, x_hi=x_hi,
                            request_id=request_id, want=("l0", "l1", "l2"))
            bufs.append(b)
            sched.append(target)
            kinds.append(k)
            tickets.append(ctx.submit(b, params))
        for t in tickets:
            done, rc = ctx.wait(t)
            assert done and rc == 0, cso.cso_last_error()
        done_t = np.array([cso.cso_ticket_times(ctx.h, t)[2] for t in tickets])
        ctx.close()
        lat = (done_t - np.array(sched)) * 1e3
        kinds = np.array(kinds)
        sl = kinds >= 0
        away = kinds >= 1  # slab 0 waits for the periodic seam, which closes with the last slab
        span = done_t[sl].max() - min(sched)
        out = {"slabs": int(sl.sum()), "particles": n, "particles_per_s": n / span,
               "p50_ms": float(np.percentile(lat[sl], 50)), "p99_ms": float(np.percentile(lat[sl], 99)),
               "p50_ms_away_from_seam": float(np.percentile(lat[away], 50)),
               "p99_ms_away_from_seam": float(np.percentile(lat[away], 99)),
               "arrivals": ("Poisson, mean gap %.0f ms" % 20) if gaps is not None else "all at t = 0"}
        if (~sl).any():
            out["small_boxes"] = {"requests": int((~sl).sum()), "p50_ms": float(np.percentile(lat[~sl], 50)),
                                  "p99_ms": float(np.percentile(lat[~sl], 99))}
        return out, [b for b, kk in zip(bufs, kinds) if kk >= 0]

    one_pass("warm-up", None, 9000)
    poisson = one_pass("poisson", rng.exponential(0.020, len(slabs)), 9001)[0]
    saturated, sbufs = one_pass("saturated", None, 9002)
    whole = None
    equal = None
    if name == "served512":
        dpos = torch.cat([s[0] for s in slabs])
        dids = torch.cat([s[1] for s in slabs])
        whole = {}
        for sched_name, fl in (("batched", cso.FLAG_BATCHED), ("plain", 0)):
            c = cso.Context(local, flags=fl)
            b = cso.Buffers(dpos, dids, True, halo_cap=n // 20 + 64, want=("l0", "l1", "l2"))
            cso.cso_find_groups(c.h, b, params)  # warm-up (workspace)
            ms = []
            for _ in range(3):
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                st = torch.cuda.ExternalStream(cso.cso_stream(c.h))
                e0.record(st)
                cso.cso_find_groups(c.h, b, params)
                e1.record(st)
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            whole[sched_name] = {"ms": statistics.median(ms), "particles_per_s": n / (statistics.median(ms) / 1e3)}
            if sched_name == "batched":
                off, equal = 0, True
                for sb in sbufs:
                    m = sb.n
                    for key in ("l0", "l1", "l2"):
                        equal = equal and bool(torch.equal(sb.out[key], b.out[key][off:off + m]))
                    off += m
            c.close()
            del b
    peaks, _ = load_peaks()
    line = {
        "metric": "CompaSO particles/s (whole hot path: density, L0, L1, L2, catalogue)",
        "value": saturated["particles_per_s"], "unit": "particles/s", "n_gpus": 1, "steps": 1, "warmup": 1,
        "ms_per_step": n / saturated["particles_per_s"] * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": name, "desc": spec["desc"], "n_particles": n, "slabs": len(slabs),
                   "budget_gb": spec["budget_gb"], "generation_s": gen_s, "seed": box.seed,
                   "l2_flush": "working set > L2 (slabs of 2-8M particles, inputs %.1f GB)" % (n * 20 / 1e9)},
        "e2e": None, "served": {"poisson": poisson, "saturated": saturated},
        "whole_box": whole, "stream_equals_whole_box": equal,
    }
    if emit:
        print(json.dumps(line), flush=True)
    return line


def radial_stage(cso, local, flags, dpos, dids, params, steps):
    """Radial statistics (r_25/50/75/98 and V_max about the L2max com) of every
    L1 halo of the benchmark box: device time of the radial stage alone (an
    optional output, outside the timed hot path), median over `steps` runs."""
    c = cso.Context(local, flags=flags | cso.FLAG_TIMING)
    b = cso.Buffers(dpos, dids, True, want=("l1", "radial"))
    for _ in range(2):
        cso.cso_find_groups(c.h, b, params)
    ms = []
    for _ in range(max(steps, 3)):
        cso.cso_find_groups(c.h, b, params)
        ms.append(cso.cso_stage_times(c.h)["radial"])
    members = int((b.out["l1"] != -1).sum().item())
    st = cso.cso_last_stats(c.h)
    c.close()
    med = statistics.median(ms)
    return {"ms": med, "l1_haloes": st["l1_nuclei"], "catalogue_rows": int(b.cout.n_halos), "l1_members": members,
            "members_per_s": members / (med / 1e3)}


def _oracle_box(args):
    side, seed = args
    import oracle as O
    from paper_2110_11408_gb300 import synth
    pos, ids, meta = synth.medium_sample(side=side, seed=seed)
    p = O.params(meta["u"])
    t0 = time.perf_counter()
    O.find_groups(pos, ids, p)
    return len(pos), time.perf_counter() - t0


def cpu_oracle_rate_all_cores(side=64, base_seed=None):
    """The oracle as it stands, one independent box per host core in parallel
    processes (the paper's embarrassingly parallel CPU layout): whole-job rate
    over the wall time of the slowest process."""
    import multiprocessing as mp
    from paper_2110_11408_gb300 import synth
    cores = os.cpu_count() or 1
    seeds = [(side, (base_seed or synth.SEED0 + 40) + k) for k in range(cores)]
    import oracle as O
    O.build()  # compile once before the workers load it
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_box, seeds)
    wall = time.perf_counter() - t0
    n_tot = sum(r[0] for r in res)
    return n_tot / wall, n_tot, wall, cores


def cpu_oracle_rate(samples):
    """Oracle (single thread) on bounded samples of the medium recipe."""
    import oracle as O
    from paper_2110_11408_gb300 import synth
    n_tot, t_tot = 0, 0.0
    for side, seed in samples:
        pos, ids, meta = synth.medium_sample(side=side, seed=seed)
        p = O.params(meta["u"])
        t0 = time.perf_counter()
        O.find_groups(pos, ids, p)
        t_tot += time.perf_counter() - t0
        n_tot += len(pos)
    return n_tot / t_tot, n_tot, t_tot


def run_reference(args, ws, rank):
    if rank != 0:
        return
    from paper_2110_11408_gb300 import synth
    import oracle as O
    times, n_tot = [], 0
    for k in range(args.warmup + args.steps):
        pos, ids, meta = synth.medium_sample(side=32, seed=synth.SEED0 + 500 + k)
        p = O.params(meta["u"])
        t0 = time.perf_counter()
        O.find_groups(pos, ids, p)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
            n_tot += len(pos)
    tot = sum(times)
    value = n_tot / tot
    sample = ("medium recipe (40% background, 60% NFW haloes N in [20, 2e5], 10% satellites) in periodic boxes of "
              "side 32 l_mean (32,768 particles), one seeded box per step")
    line = {"impl": "reference", "metric": "CompaSO particles/s (whole hot path: density, L0, L1, L2, catalogue)",
            "value": value, "unit": "particles/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * tot / len(times), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int64", "data": "synthetic", "config": {"workload": args.workload, "sample": sample},
            "cpu_baseline": {"value": value, "unit": "particles/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "particles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="medium", choices=sorted(WORKLOADS) + sorted(SERVED_SCALE))
    ap.add_argument("--plain", action="store_true", help="time the plain schedule as the headline (default: batched)")
    ap.add_argument("--no-compare", action="store_true", help="skip timing the other schedule")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--bins", default="", help="giant,small size bins of the batched schedule instead of autotuning")
    ap.add_argument("--huge", type=int, default=0, help="groups above this many members on 16-CTA clusters (0: library default)")
    ap.add_argument("--no-radial", action="store_true", help="skip timing the radial statistics stage")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    ws, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, ws, rank)

    import torch
    from paper_2110_11408_gb300 import cso

    torch.cuda.set_device(local)
    if args.workload in SERVED_SCALE:
        return served_at_scale(args, cso, torch, local, args.workload)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    # CPU baseline first (before any device context gets forked around)
    cpu = cpu_all = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        from paper_2110_11408_gb300 import synth
        rate, n_cpu, t_cpu = cpu_oracle_rate([(64, synth.SEED0 + 21), (64, synth.SEED0 + 22)])
        cpu = {"value": rate, "unit": "particles/s", "cores": 1, "kind": "oracle",
               "sample": "medium recipe in two seeded periodic boxes of side 64 l_mean (2 x 262,144 particles), "
                         "%.1f s of single-thread oracle time" % t_cpu}
        rate_all, n_all, wall_all, cores = cpu_oracle_rate_all_cores()
        cpu_all = {"value": rate_all, "unit": "particles/s", "cores": cores, "kind": "oracle",
                   "sample": "medium recipe, %d seeded periodic boxes of side 64 l_mean (one per core, %d particles "
                             "in all) in parallel processes, %.1f s wall" % (cores, n_all, wall_all)}

    # measured pipe rates of this GPU (integer ALU, IMAD, shared-memory
    # broadcast), the denominators of the pair-kernel roofline
    pipes = cso.cso_probe_peaks(local) if rank == 0 else None

    pos, ids, meta = make_workload(args.workload, rank)
    n = len(pos)
    params = cso.cso_params_default(meta["u"])
    primary = "plain" if args.plain else "batched"
    flags = cso.FLAG_TIMING | (0 if args.plain else cso.FLAG_BATCHED)
    dpos = torch.from_numpy(pos).cuda()
    dids = torch.from_numpy(ids.view(np.int64)).cuda()
    buf = cso.Buffers(dpos, dids, on_device=True)
    torch.cuda.synchronize()

    # algorithmic pair count of this box (untimed pass with the counter on)
    cctx = cso.Context(local, flags=cso.FLAG_COUNT_PAIRS)
    cso.cso_find_groups(cctx.h, buf, params)
    stats = cso.cso_last_stats(cctx.h)
    cctx.close()

    tuned = None

    def time_schedule(fl, clk=None):
        nonlocal tuned
        c = cso.Context(local, flags=fl)
        if fl & cso.FLAG_BATCHED:
            if args.bins:  # fixed size bins (profiling runs)
                g_, s_ = (int(v) for v in args.bins.split(","))
                cso.cso_set_schedule(c.h, g_, s_)
                tuned = (g_, s_)
            else:  # size bins picked by the autotuner on this machine (untimed)
                tuned = cso.cso_autotune(c.h, buf, params)
            if args.huge:
                cso.cso_set_huge_group(c.h, args.huge)
        stream = torch.cuda.ExternalStream(cso.cso_stream(c.h))
        for _ in range(args.warmup):
            cso.cso_find_groups(c.h, buf, params)
        torch.cuda.synchronize()
        barrier()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        acc = {}
        if clk:
            clk.__enter__()
        torch.cuda.synchronize()
        if clk:
            clk.mark(0)
        ev0.record(stream)
        for _ in range(args.steps):
            cso.cso_find_groups(c.h, buf, params)
            for k, v in cso.cso_stage_times(c.h).items():
                acc.setdefault(k, []).append(v)
        ev1.record(stream)
        torch.cuda.synchronize()
        if clk:
            clk.mark(1)
            clk.__exit__()
        barrier()
        t = ev0.elapsed_time(ev1) / args.steps
        st = cso.cso_last_stats(c.h)
        _, t = whole_job_rate(n, t, ws, dist, "cuda")
        return c, t, acc, st

    clk = ClockSampler(local)
    ctx, ms, stage_acc, stats_t = time_schedule(flags, clk)
    value = ws * n / (ms / 1e3)
    other = None
    if not args.no_compare:
        c2, ms2, _, _ = time_schedule(cso.FLAG_TIMING | (cso.FLAG_BATCHED if args.plain else 0))
        c2.close()
        other = {"schedule": "batched" if args.plain else "plain", "value": ws * n / (ms2 / 1e3),
                 "ms_per_step": ms2}

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        hpos = torch.from_numpy(pos).pin_memory()
        hids = torch.from_numpy(ids.view(np.int64)).pin_memory()
        hp, hi = hpos.numpy(), hids.numpy().view(np.uint64)
        hb = cso.Buffers(hp, hi, on_device=False)
        for name in list(hb.out):
            hb.out[name] = torch.empty(n, dtype=torch.int64).pin_memory().numpy().view(
                np.int64 if name == "sigma" else np.uint64)
        hb.halos = torch.empty(hb.halo_cap * cso.HALO_DTYPE.itemsize, dtype=torch.uint8).pin_memory().numpy().view(
            cso.HALO_DTYPE)
        hb.cout = cso.CsoOutput(l0=hb.out["l0"].ctypes.data, l1=hb.out["l1"].ctypes.data,
                                l2=hb.out["l2"].ctypes.data, sigma=hb.out["sigma"].ctypes.data,
                                halos=hb.halos.ctypes.data, halo_cap=hb.halo_cap, n_halos=0, on_device=0)
        for _ in range(2):
            cso.cso_find_groups(ctx.h, hb, params)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            cso.cso_find_groups(ctx.h, hb, params)
            _ = int(hb.cout.n_halos)
        dt = (time.perf_counter() - t0) / args.steps
        _, ms_e2e = whole_job_rate(n, dt * 1e3, ws, dist, "cuda")
        dt = ms_e2e / 1e3
        h2d = n * (12 + 8)
        d2h = n * 8 * 4 + int(hb.cout.n_halos) * cso.HALO_DTYPE.itemsize
        e2e = {"value": ws * n / dt, "unit": "particles/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    # the batched step with its CompaSO level stages replayed as captured
    # CUDA graphs, against direct launches
    graph = None
    if not args.no_compare and ws == 1 and not args.plain:
        def step_ms(fl):
            c4 = cso.Context(local, flags=fl)
            if tuned:
                cso.cso_set_schedule(c4.h, tuned[0], tuned[1])
            s4 = torch.cuda.ExternalStream(cso.cso_stream(c4.h))
            for _ in range(args.warmup):
                cso.cso_find_groups(c4.h, buf, params)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s4)
            for _ in range(args.steps):
                cso.cso_find_groups(c4.h, buf, params)
            e1.record(s4)
            torch.cuda.synchronize()
            c4.close()
            return e0.elapsed_time(e1) / args.steps
        base_fl = cso.FLAG_BATCHED
        graph = {"ms_per_step_direct": step_ms(base_fl), "ms_per_step_graph": step_ms(base_fl | cso.FLAG_GRAPH)}

    # the paper's radial-bin threshold-radius search against the default
    # threshold-count binning: device time of the CompaSO level stages
    r_search = None
    if not args.no_compare and ws == 1:
        r_search = {}
        for label, fl in (("threshold_count_bins", 0), ("radial_bins", cso.FLAG_RADIAL_BINS)):
            c3 = cso.Context(local, flags=flags | fl)
            if tuned:
                cso.cso_set_schedule(c3.h, tuned[0], tuned[1])
            lv = []
            for rep in range(args.warmup + args.steps):
                cso.cso_find_groups(c3.h, buf, params)
                st3 = cso.cso_stage_times(c3.h)
                if rep >= args.warmup:
                    lv.append(st3.get("level1", 0.0) + st3.get("level2", 0.0))
            c3.close()
            r_search[label + "_levels_ms"] = statistics.median(lv)

    radial = None
    if not args.no_radial and ws == 1:
        radial = radial_stage(cso, local, flags & ~cso.FLAG_TIMING, dpos, dids, params, args.steps)

    served = None
    if not args.no_served and ws == 1:
        served = {"boxes": served_stream(cso, torch, local, flags & ~cso.FLAG_TIMING),
                  "slab_stream": slab_stream(cso, torch, local, flags & ~cso.FLAG_TIMING, pos, ids, meta)}
        if args.workload == "medium":
            # the served configuration of side 512 (134M particles in 64 slabs)
            s5 = served_at_scale(args, cso, torch, local, "served512", emit=False)
            served["served512"] = {"desc": s5["config"]["desc"], "n_particles": s5["config"]["n_particles"],
                                   "stream": s5["served"], "whole_box": s5["whole_box"],
                                   "stream_equals_whole_box": s5["stream_equals_whole_box"]}
            torch.cuda.empty_cache()

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    stages = {k: statistics.median(v) for k, v in stage_acc.items()}
    peaks, peak_src = load_peaks()
    clocks = clk.summary()
    # dominant kernel: the density pair loop, bounded by the integer ALU
    dens_ms = stages.get("density")
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    n_sms = torch.cuda.get_device_properties(local).multi_processor_count
    derived_peak = n_sms * 128 * sm_mhz * 1e6 / 1e12  # int32 lane-ops / s, in T/s
    alu_peak = pipes["alu_tops"] if pipes else derived_peak
    roof = None
    if dens_ms:
        achieved = stats["pairs_b"] * OPS_PER_PAIR / (dens_ms / 1e3) / 1e12
        roof = {"bound": "alu", "kernel": "k_density", "achieved": achieved, "peak": alu_peak,
                "unit": "Tops/s", "frac": achieved / alu_peak,
                "traffic": DENSITY_DRAM_BYTES.get(args.workload),
                "peak_source": ("measured: integer add/xor lane-op chains on this GPU (cso_probe_peaks)" if pipes
                                else "derived: %d SMs x 128 int32 lanes x %.0f MHz" % (n_sms, sm_mhz)),
                "peak_derived": derived_peak, "pipes": pipes,
                "algorithmic": "%d pairs within b x %d int ops" % (stats["pairs_b"], OPS_PER_PAIR)}
    line = {
        "metric": "CompaSO particles/s (whole hot path: density, L0, L1, L2, catalogue)",
        "value": value, "unit": "particles/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic",
        "config": {"workload": args.workload, "desc": WORKLOADS[args.workload]["desc"], "n_particles": n,
                   "schedule": primary, "autotuned_bins": tuned, "l2_flush": "working set > L2 (inputs %.0f MB, cell table %.2f GB, L2 129 MB)"
                   % (n * 20 / 1e6, cell_table_bytes(meta["u"]) / 1e9), "seed": meta["seed"]},
        "e2e": e2e, "gpu_launches": stats_t["launches"] * args.steps, "roofline": roof, "cpu_baseline": cpu,
        "cpu_baseline_all_cores": cpu_all, "clocks": clocks, "served": served, "other_schedule": other,
        "radial": radial, "r_search": r_search, "level_graph": graph,
        "stages_ms": stages,
        "counts": {k: stats[k] for k in ("dense", "l0_groups", "l1_nuclei", "l2_nuclei", "catalogue_rows",
                                         "pairs_b", "l1_work", "l2_work", "workspace_bytes")},
    }
    print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
