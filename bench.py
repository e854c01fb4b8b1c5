"""Benchmark of the coupled-configuration hot path on GB300.

One step = count -> scan -> fill -> de-duplicate over one batch of sources of the
mid-size system (52 spin orbitals, 7 alpha + 7 beta electrons, 100k sources
drawn as random excitations of rank <= 4 out of the aufbau determinant,
eps = 1e-8).  The metric is entries per second: coupled entries surviving the
screening (diagonal included) generated and de-duplicated per second.  The
energy forward + adjoint over a 200k selected set of the same system is timed
beside it and reported as ``energy_fwd_bwd_ms``.

``--impl reference`` times the CPU oracle instead, on a bounded sample of the
same workload, on this host's cores.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank runs an independent replica of the workload
(the path is not sharded), the time is the maximum over ranks and the value the
sum of all ranks' entries over that time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "coupled configs (+H_ij) generated & deduped per sec; % HBM roofline; energy+grad ms"

# DRAM bytes per entry (dram__bytes_read.sum + dram__bytes_write.sum) of each
# C-ABI call, from one ncu capture of the first 20k sources of the same
# workload (profiles/traffic_mid_20k.md), scaled to a launch by its entries.
# Set an entry to None when the kernels behind it change before a re-capture.
WORKLOADS = {
    "mid": "mid: 52 spin orbitals, 7a+7b electrons, {n} sources (random excitations of "
           "rank<=4), eps=1e-8",
    "tiny": "tiny: 16 spin orbitals, 4a+4b electrons, all {n} determinants of the FCI space, "
            "eps=0",
    "large": "large: 120 spin orbitals (2 words), 10a+10b electrons, {n} sources, eps=1e-6, "
             "in HBM (no streaming)",
}

TRAFFIC_B_PER_ENTRY = {"cusci_dedup": 117.15, "cusci_gen_coupled (fill_kernel)": 15.93}
# the same capture per phase of the dedup call (the phase names of
# cusci_dedup_phase_name; scans and tiny launches folded into their phase)
DEDUP_KERNEL_B_PER_ENTRY = {"sample+splitters": 1.93, "hist1": 9.95, "scatter1": 24.21,
                            "level2": 32.80, "leaf_dedup": 14.54, "compact_unique": 4.99,
                            "unscatter2": 16.84, "unscatter1": 11.90}
UNIT = "entries/s"


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        fd, self.path = tempfile.mkstemp(prefix="cusci_clocks_", suffix=".csv")
        os.close(fd)

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None or not os.path.exists(self.path):
            out["reasons"] = ["nvidia-smi unavailable"]
            return out
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if sm:
            out.update(sm_mhz=statistics.median(sm), sm_max_mhz=max(smax), samples=len(sm))
        out["reasons"] = sorted(reasons)
        try:
            os.unlink(self.path)
        except OSError:
            pass
        return out


def aggregate_over_ranks(ms_local: float, entries_local: int, device=None):
    """Whole-job figures of independent replicas: the slowest rank's time and the
    sum of all ranks' entries (plain values when not distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms_local, entries_local
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    e = torch.tensor([entries_local], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(e, op=dist.ReduceOp.SUM)
    return float(t.item()), int(e.item())


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ----------------------------------------------------------------------------- reference arm
def run_reference(args):
    """The CPU oracle on a bounded sample of the workload (this host's cores)."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    from oracle import oracle as O
    from paper_2604_15768_gb300 import synth
    s = synth.config_system(args.workload, n_dets=ref_sample(args))
    osys = O.OracleSystem.of(s)
    times, entries = [], 0
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        counts = osys.count(s.dets, s.eps)
        off, td, hv = osys.gen(s.dets, s.eps, counts)
        u, inv = O.dedup(td)
        dt = time.perf_counter() - t0
        entries = int(off[-1])
        if it >= args.warmup:
            times.append(dt)
    t = float(np.mean(times))
    value = entries / t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload].format(n=s.dets.shape[0])
                   + " (bounded CPU sample: the first sources of the workload)",
                   "sources": int(s.dets.shape[0]), "entries_per_step": entries},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.threads(), "kind": "oracle",
                         "sample": f"first {s.dets.shape[0]} sources of the {args.workload} "
                                   "workload, count+gen+dedup"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- our arm
def run_ours(args):
    import torch

    from paper_2604_15768_gb300 import cusci, synth

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    hbm_peak, peak_kind = _peaks()

    s = synth.config_system(args.workload, n_dets=args.sources)
    sysd = cusci.System.of(s)
    n, W = s.dets.shape
    n_bits, n_ones = 2 * s.norb, s.n_alpha + s.n_beta
    d_src = cusci.dets_to_device(s.dets, dev)
    stream = torch.cuda.current_stream()

    # sizes from one untimed pass
    counts = cusci.count_coupled(sysd, d_src, s.eps)
    offsets = cusci.exclusive_scan(counts)
    total = int(offsets[-1].item())
    idx_bytes = 4 if total < 2 ** 31 else 8
    out_d = torch.empty((total, W), dtype=torch.int64, device=dev)
    out_h = torch.empty(total, dtype=torch.float64, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    scan_ws = torch.empty(cusci.scan_workspace(n), dtype=torch.uint8, device=dev)
    dd_ws = torch.empty(cusci.dedup_workspace(total, W, n_bits, n_ones), dtype=torch.uint8,
                        device=dev)
    uniq = torch.empty((total, W), dtype=torch.int64, device=dev)
    inv = torch.empty(total, dtype=torch.int32 if idx_bytes == 4 else torch.int64, device=dev)
    d_nu = torch.zeros(1, dtype=torch.int64, device=dev)
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device=dev)

    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def step(marks=None):
        m = marks or [None] * 4
        cusci.count_coupled(sysd, d_src, s.eps, out=counts)
        cusci.exclusive_scan(counts, out=offsets, workspace=scan_ws)
        if m[1] is not None:
            m[1].record(stream)
        cusci.gen_coupled(sysd, d_src, s.eps, offsets, total, out_dets=out_d, out_h=out_h,
                          status=status)
        if m[2] is not None:
            m[2].record(stream)
        cusci.dedup_into(out_d, n_bits, n_ones, uniq, inv, d_nu, dd_ws)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    n_unique = int(d_nu.item())
    assert int(status.item()) == 0, "fill pass reported inconsistent offsets"

    l0 = cusci.kernel_launches()
    per_step, t_count, t_gen, t_dedup = [], [], [], []
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    cusci.set_kernel_timing(True)   # per-phase events inside the dedup calls of the timed steps
    wall0 = time.perf_counter()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()                               # L2 flush, outside the events
            marks = [ev(), ev(), ev(), ev()]
            marks[0].record(stream)
            step(marks)
            marks[3].record(stream)
            per_step.append(marks)
        torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    launches = cusci.kernel_launches() - l0
    phase_ms, phase_calls = cusci.dedup_phase_ms()
    cusci.set_kernel_timing(False)
    for m in per_step:
        t_count.append(m[0].elapsed_time(m[1]))
        t_gen.append(m[1].elapsed_time(m[2]))
        t_dedup.append(m[2].elapsed_time(m[3]))
    step_ms = [a + b + c for a, b, c in zip(t_count, t_gen, t_dedup)]
    ms = float(np.mean(step_ms))
    ms, job_entries = aggregate_over_ranks(ms, total, device=dev)
    if ws > 1:
        torch.distributed.barrier()
    value = job_entries / (ms * 1e-3)

    # algorithmic bytes (8W+8 written per entry by the fill, 8W read + inverse
    # written per entry and 8W per distinct key by the dedup, 8W + 16 per source)
    gen_bytes = total * (8 * W + 8) + n * (8 * W + 16)
    dedup_bytes = total * (8 * W + idx_bytes) + n_unique * 8 * W
    step_bytes = gen_bytes + dedup_bytes + n * 16
    gen_ms, dedup_ms, count_ms = (float(np.mean(t_gen)), float(np.mean(t_dedup)),
                                  float(np.mean(t_count)))
    gen_gbs = gen_bytes / (gen_ms * 1e-3) / 1e9
    dedup_gbs = dedup_bytes / (dedup_ms * 1e-3) / 1e9
    dominant = "cusci_dedup" if dedup_ms >= gen_ms else "cusci_gen_coupled (fill_kernel)"
    tpe = TRAFFIC_B_PER_ENTRY.get(dominant) if args.workload == "mid" else None
    traffic = None if tpe is None else tpe * total
    # the dedup call's kernels: mean CUDA-event time per call over the timed
    # steps, DRAM traffic per launch from the capture, achieved DRAM GB/s
    hbm_peak_k, _ = _peaks()
    dedup_kernels = {}
    for name, tot_ms in phase_ms.items():
        if phase_calls == 0:
            break
        k_ms = tot_ms / phase_calls
        bpe = DEDUP_KERNEL_B_PER_ENTRY.get(name) if args.workload == "mid" else None
        rec = {"ms": k_ms}
        if bpe is not None and k_ms > 0:
            gbs = bpe * total / (k_ms * 1e-3) / 1e9
            rec.update({"dram_b_per_entry": bpe, "dram_gbs": gbs, "frac_of_hbm": gbs / hbm_peak_k})
        dedup_kernels[name] = rec
    dom_gbs, dom_bytes, dom_ms = ((dedup_gbs, dedup_bytes, dedup_ms) if dedup_ms >= gen_ms
                                  else (gen_gbs, gen_bytes, gen_ms))

    # the paper's distributed de-duplication (Sec. 4.1.1) over virtual ranks:
    # load balance (Max/Min, CV of distinct items per rank) and throughput
    ranks = None
    if args.ranks:
        del dd_ws
        dd_ws = None
        torch.cuda.empty_cache()
        off_h = offsets.cpu().numpy()
        ranks = {}
        for P, S in ((8, 1024), (64, 256)):
            eo = off_h[np.linspace(0, n, P + 1).astype(np.int64)]
            for _ in range(2):  # the first run warms the allocator; the second is timed
                parts = None
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                parts, st_r, _, _, _, _ = cusci.virtual_rank_dedup(out_d, eo, P, S, n_bits,
                                                                   n_ones)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
            ranks[f"P{P}"] = {"max_over_min": st_r["max_over_min"], "cv": st_r["cv"],
                              "unique_max_over_min": st_r["unique_max_over_min"],
                              "unique_cv": st_r["unique_cv"],
                              "ms": dt * 1e3, "M_items_per_s": total / dt / 1e6,
                              "distinct_total": int(sum(st_r["unique"]))}
            del parts
            torch.cuda.empty_cache()
        ranks["workload"] = ("mid step's coupled set split by contiguous source ranges over P "
                             "virtual ranks; max_over_min / cv of the items each rank holds "
                             "after the exchange (the paper's metric), unique_* of its distinct "
                             "keys; ms: the whole device pipeline (rank join, one dedup for "
                             "Step 1, plan, exchange gather, one dedup for the final merge, "
                             "split) including its allocations and one host read-back")

    # local-energy form (Eq. 5) over this step's coupled lists and reverse index,
    # with synthetic amplitudes on the distinct set
    loc = None
    if args.energy:
        out_d = dd_ws = uniq = None
        torch.cuda.empty_cache()
        gpsi = torch.Generator(device=dev).manual_seed(7)
        psi_u = 1.0 + 0.1 * torch.randn(n_unique, dtype=torch.float64, device=dev, generator=gpsi)
        lws = torch.empty(cusci.local_energy_workspace(n), dtype=torch.uint8, device=dev)
        invv = inv[:total]
        for _ in range(2):
            E_l, n2_l, y_l = cusci.local_energy_fwd(offsets, out_h, invv, psi_u, workspace=lws)
            g_l = cusci.local_energy_bwd(offsets, out_h, invv, psi_u, E_l, n2_l, y=y_l)
        fw, bw = [], []
        for _ in range(3):
            a0, a1, a2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            a0.record()
            E_l, n2_l, y_l = cusci.local_energy_fwd(offsets, out_h, invv, psi_u, workspace=lws)
            a1.record()
            g_l = cusci.local_energy_bwd(offsets, out_h, invv, psi_u, E_l, n2_l, y=y_l)
            a2.record()
            torch.cuda.synchronize()
            fw.append(a0.elapsed_time(a1))
            bw.append(a1.elapsed_time(a2))
        f_ms, b_ms = float(np.median(fw)), float(np.median(bw))
        alg = total * (8 + idx_bytes + 8) + n * 16
        loc = {"fwd_ms": f_ms, "bwd_ms": b_ms, "fwd_bwd_ms": f_ms + b_ms, "E": float(E_l.item()),
               "entries": total, "distinct": n_unique,
               "fwd_algorithmic_gbs": alg / (f_ms * 1e-3) / 1e9,
               "fwd_frac_of_hbm": alg / (f_ms * 1e-3) / 1e9 / hbm_peak,
               "workload": "Eq. 5 local form over the timed step's coupled lists; psi on the "
                           "distinct set = 1 + 0.1 N(0,1), seeded"}
        # streaming two-level top-K over the distinct set by |psi| (Stage 2)
        K_top, tb = 100_000, 16_000_000
        tk = cusci.TopK(K_top, tb)
        ids_all = torch.arange(n_unique, dtype=torch.int64, device=dev)
        score_all = psi_u.abs()
        for a_ in range(0, n_unique, tb):
            tk.update(score_all[a_:a_ + tb], ids_all[a_:a_ + tb])
        tk.count.zero_()
        torch.cuda.synchronize()
        k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k0.record()
        for a_ in range(0, n_unique, tb):
            tk.update(score_all[a_:a_ + tb], ids_all[a_:a_ + tb])
        k1.record()
        torch.cuda.synchronize()
        tk_ms = k0.elapsed_time(k1)
        loc["topk"] = {"K": K_top, "batch": tb, "items": n_unique, "ms": tk_ms,
                       "items_per_s": n_unique / (tk_ms * 1e-3),
                       "kept": int(tk.count.item())}
        del psi_u, lws, g_l, y_l, tk, ids_all, score_all

    # release the timed step's buffers before the other measurements
    out_d = out_h = dd_ws = uniq = inv = flush = None
    torch.cuda.empty_cache()

    # end to end through the public API with host buffers
    e2e = run_e2e(args, s, sysd, dev) if args.e2e else None
    if e2e is not None and ws > 1:
        # whole job: every rank's entries over the slowest rank's step
        e_ms, e_entries = aggregate_over_ranks(e2e["ms_per_step"], total, device=dev)
        e2e.update({"value": e_entries / (e_ms * 1e-3), "ms_per_step": e_ms,
                    "h2d_bytes_per_step": e2e["h2d_bytes_per_step"] * ws,
                    "d2h_bytes_per_step": e2e["d2h_bytes_per_step"] * ws})
    torch.cuda.empty_cache()

    # energy forward + adjoint on the 200k selected set
    energy = run_energy(args, dev) if args.energy else None

    torch.cuda.empty_cache()
    stream_res = run_stream(args, dev) if args.stream else None
    torch.cuda.empty_cache()
    batch_res = run_batched(args, dev) if args.batched else None
    torch.cuda.empty_cache()

    # CPU oracle on a bounded sample (rank 0, N = 1 only)
    cpu = run_cpu_baseline(args) if (rank == 0 and ws == 1 and args.cpu_baseline) else None

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64+f64",
            "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload].format(n=n),
                       "sources": n, "entries_per_step": total, "unique_per_step": n_unique,
                       "inverse_bytes": idx_bytes, "parallelism": f"replicas{ws}",
                       "l2": "flushed between steps (256 MiB write outside the timed events); "
                             "each step also moves >40 GB"},
            "roofline": {"bound": "hbm", "achieved": dom_gbs, "peak": hbm_peak, "unit": "GB/s",
                         "frac": dom_gbs / hbm_peak, "traffic": traffic, "kernel": dominant,
                         "algorithmic_bytes_per_launch": dom_bytes, "ms_per_launch": dom_ms,
                         "peak_kind": f"{peak_kind} (copy, burst)"},
            "step_roofline": {"algorithmic_bytes": step_bytes,
                              "achieved_gbs": step_bytes / (ms * 1e-3) / 1e9,
                              "frac": step_bytes / (ms * 1e-3) / 1e9 / hbm_peak},
            "phases_ms": {"count+scan": count_ms, "gen": gen_ms, "dedup": dedup_ms},
            "dedup_kernels": dedup_kernels,
            "phases_gbs": {"gen": gen_gbs, "dedup": dedup_gbs},
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "wall_s_timed": wall,
        }
        if e2e is not None:
            line["e2e"] = e2e
        if energy is not None:
            line["energy_fwd_bwd_ms"] = energy["fwd_bwd_ms"]
            line["energy"] = energy
        if loc is not None:
            line["local_energy"] = loc
        if ranks is not None:
            line["virtual_ranks"] = ranks
        if cpu is not None:
            line["cpu_baseline"] = cpu
        if stream_res is not None:
            line["streaming"] = stream_res
        if batch_res is not None:
            line["batched"] = batch_res
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_e2e(args, s, sysd, dev):
    """Same metric through the public API with host buffers: every step copies
    the sources in from pinned host memory, runs count/scan/fill/dedup, and
    copies the step's result -- the sorted distinct targets and the reverse
    index of every coupled entry -- back to pinned host memory."""
    import torch

    from paper_2604_15768_gb300 import cusci
    host = torch.from_numpy(np.ascontiguousarray(s.dets).view(np.int64)).pin_memory()
    n_bits, n_ones = 2 * s.norb, s.n_alpha + s.n_beta
    W = s.dets.shape[1]
    # sizes of the result (deterministic: the same every step)
    d = host.to(dev)
    off, od, oh, st = cusci.coupled(sysd, d, s.eps)
    u, inv, nu = cusci.dedup(od, n_bits, n_ones)
    total, n_unique = int(od.shape[0]), int(nu)
    del d, off, od, oh, st, u, inv
    torch.cuda.empty_cache()
    h_unique = torch.empty((n_unique, W), dtype=torch.int64).pin_memory()
    h_inverse = torch.empty(total, dtype=torch.int32 if total < 2 ** 31 else torch.int64).pin_memory()
    times = []
    parts = []

    def one():
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        ev[0].record()
        d = host.to(dev, non_blocking=True)
        ev[1].record()
        off, od, oh, st = cusci.coupled(sysd, d, s.eps)
        ev[2].record()
        u, inv, d_nu = cusci.dedup(od, n_bits, n_ones, sync=False)
        ev[3].record()
        h_unique.copy_(u[:n_unique], non_blocking=True)
        ev[4].record()
        h_inverse.copy_(inv, non_blocking=True)
        ev[5].record()
        torch.cuda.current_stream().synchronize()
        return int(od.shape[0]), [ev[i].elapsed_time(ev[i + 1]) for i in range(5)]

    for _ in range(2):
        one()
    for _ in range(max(2, args.steps // 2)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        got, ph = one()
        times.append(time.perf_counter() - t0)
        parts.append(ph)
        assert got == total
    t = float(np.mean(times))
    ph = np.mean(np.array(parts), axis=0)
    # yardstick: a plain copy of the inverse's bytes from a fresh device
    # buffer into the same pinned buffer
    src = torch.empty_like(h_inverse, device=dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(2):
        torch.cuda.synchronize()
        a.record()
        h_inverse.copy_(src, non_blocking=True)
        b.record()
        torch.cuda.synchronize()
    yard = h_inverse.numel() * h_inverse.element_size() / (a.elapsed_time(b) * 1e-3) / 1e9
    del src
    d2h = int(h_unique.numel() * 8 + h_inverse.numel() * h_inverse.element_size())
    serial = {"ms_per_step": t * 1e3, "value": total / t,
              "phases_ms": {"h2d": float(ph[0]), "count+scan+fill": float(ph[1]),
                            "dedup": float(ph[2]), "d2h_unique": float(ph[3]),
                            "d2h_inverse": float(ph[4])},
              "d2h_gbs": d2h / (float(ph[3] + ph[4]) * 1e-3) / 1e9 if ph[3] + ph[4] > 0 else None,
              "api": "cusci.coupled + cusci.dedup, one step at a time"}
    del h_unique, h_inverse
    torch.cuda.empty_cache()
    tp = _e2e_pipelined(args, s, sysd, dev, host, total, n_unique)
    return {"value": total / tp, "unit": UNIT, "h2d_bytes_per_step": int(host.numel() * 8),
            "d2h_bytes_per_step": d2h, "ms_per_step": tp * 1e3, "plain_pinned_d2h_gbs": yard,
            "serial": serial,
            "api": "cusci.count_coupled + exclusive_scan + gen_coupled + dedup_into, steps back "
                   "to back: every step copies its sources in from pinned host memory and its "
                   "sorted distinct set and reverse index out to pinned host memory on a side "
                   "stream, overlapped with the next step's kernels (double-buffered results)"}


def _e2e_pipelined(args, s, sysd, dev, host, total, n_unique):
    """Seconds per step of back-to-back steps through the public API, each
    step's result read back on a side stream while the next step computes:
    two result buffers on the device and on the host, the compute stream
    waiting for a buffer's read-back before reusing it."""
    import torch

    from paper_2604_15768_gb300 import cusci
    n, W = s.dets.shape
    n_bits, n_ones = 2 * s.norb, s.n_alpha + s.n_beta
    d_src = torch.empty((n, W), dtype=torch.int64, device=dev)
    counts = torch.empty(n, dtype=torch.int64, device=dev)
    offsets = torch.empty(n + 1, dtype=torch.int64, device=dev)
    scan_ws = torch.empty(cusci.scan_workspace(n), dtype=torch.uint8, device=dev)
    out_d = torch.empty((total, W), dtype=torch.int64, device=dev)
    out_h = torch.empty(total, dtype=torch.float64, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    dd_ws = torch.empty(cusci.dedup_workspace(total, W, n_bits, n_ones), dtype=torch.uint8,
                        device=dev)
    uniq = [torch.empty((total, W), dtype=torch.int64, device=dev) for _ in range(2)]
    inv = [torch.empty(total, dtype=torch.int32, device=dev) for _ in range(2)]
    d_nu = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in range(2)]
    h_u = [torch.empty((n_unique, W), dtype=torch.int64).pin_memory() for _ in range(2)]
    h_i = [torch.empty(total, dtype=torch.int32).pin_memory() for _ in range(2)]
    cs = torch.cuda.current_stream()
    xs = torch.cuda.Stream()
    done = [None, None]

    def step(k):
        b = k % 2
        if done[b] is not None:
            cs.wait_event(done[b])                 # the buffer's previous read-back left
        d_src.copy_(host.view(n, W), non_blocking=True)
        cusci.count_coupled(sysd, d_src, s.eps, out=counts)
        cusci.exclusive_scan(counts, out=offsets, workspace=scan_ws)
        cusci.gen_coupled(sysd, d_src, s.eps, offsets, total, out_dets=out_d, out_h=out_h,
                          status=status)
        cusci.dedup_into(out_d, n_bits, n_ones, uniq[b], inv[b], d_nu[b], dd_ws)
        ready = torch.cuda.Event()
        ready.record(cs)
        with torch.cuda.stream(xs):
            xs.wait_event(ready)
            h_u[b].copy_(uniq[b][:n_unique], non_blocking=True)
            h_i[b].copy_(inv[b][:total], non_blocking=True)
            done[b] = torch.cuda.Event()
            done[b].record(xs)

    for k in range(3):
        step(k)
    torch.cuda.synchronize()
    steps = max(4, args.steps)
    t0 = time.perf_counter()
    for k in range(steps):
        step(k)
    torch.cuda.synchronize()
    tp = (time.perf_counter() - t0) / steps
    assert int(status.item()) == 0 and int(d_nu[0].item()) == n_unique
    # the host copies hold this step's result: spot-check against the device
    assert torch.equal(h_i[(steps - 1) % 2][:1000], inv[(steps - 1) % 2][:1000].cpu())
    return tp


def run_energy(args, dev):
    import torch

    from paper_2604_15768_gb300 import cusci, synth
    s = synth.config_system("energy", n_dets=args.energy_sources)
    sysd = cusci.System.of(s)
    dS = cusci.dets_to_device(s.dets, dev)
    net, x = synth.amplitude_mlp(s.dets, s.norb, dev)

    def fwd_bwd():
        psi = torch.exp(net(x).squeeze(-1).double())
        E = cusci.Energy.apply(psi, sysd, dS, s.eps, False)
        E.backward()
        return E

    for _ in range(2):
        fwd_bwd()
    torch.cuda.synchronize()
    # time only the library's forward and adjoint with events
    psi = torch.exp(net(x).squeeze(-1).double()).detach()
    ws_e = torch.empty(cusci.energy_workspace(sysd, dS.shape[0]), dtype=torch.uint8, device=dev)
    fwd, bwd = [], []
    for _ in range(3):
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a.record()
        E, n2, hp = cusci.energy_fwd(sysd, dS, psi, s.eps, workspace=ws_e)
        b.record()
        cusci.energy_bwd(sysd, dS, psi, s.eps, E, n2, hpsi=hp, workspace=ws_e)
        c.record()
        torch.cuda.synchronize()
        fwd.append(a.elapsed_time(b))
        bwd.append(b.elapsed_time(c))
    return {"fwd_ms": float(np.median(fwd)), "bwd_ms": float(np.median(bwd)),
            "fwd_bwd_ms": float(np.median(fwd) + np.median(bwd)), "E": float(E.item()),
            "selected": int(dS.shape[0]),
            "workload": "mid system, selected set of sorted distinct sampled dets, psi from a "
                        "seeded 256-256 tanh MLP"}


def run_stream(args, dev):
    """Large two-word system (120 spin orbitals, 10a+10b, 20k sources, eps 1e-6)
    through mini-batches of a bounded pool, coupled lists offloaded to pinned
    host memory.  The distinct-set capacity is the measured distinct count plus
    10% (the pool then holds the hash set of the distinct keys, the two batch
    buffers and the per-source arrays); a plain pinned device-to-host copy of
    the same bytes is timed beside it, and the peak pool use is reported
    against the batch size with and without the offload (Sec. 5.6)."""
    import torch

    from paper_2604_15768_gb300 import cusci, synth
    s = synth.config_system("large", n_dets=args.stream_sources)
    sysd = cusci.System.of(s)
    batch = args.stream_batch
    # host capacity from the counts and distinct capacity from one untimed run
    d = cusci.dets_to_device(s.dets, dev)
    total = int(cusci.count_coupled(sysd, d, s.eps).sum().item())
    del d
    torch.cuda.empty_cache()
    probe = cusci.stream_gen_dedup(sysd, s.dets, s.eps, batch, total, host_capacity=total)
    n_distinct = int(probe[3].shape[0])
    del probe
    torch.cuda.empty_cache()
    ucap = int(n_distinct * 1.1) + 1024 if args.stream_unique_cap <= 0 else args.stream_unique_cap
    hcap = total
    buffers = cusci.stream_buffers(sysd, s.dets, batch, ucap, hcap)
    res = None
    times, stats = [], []
    for it in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = cusci.stream_gen_dedup(sysd, s.dets, s.eps, batch, ucap, buffers=buffers)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
        stats.append(res[4])
    off, hd, hh, uniq, _ = res
    best = 1 + int(np.argmin(times[1:]))    # the first run is a warm-up
    t, st = times[best], stats[best]
    run_ms = [round(x * 1e3, 3) for x in times[1:]]
    # yardstick: one plain pinned copy of the same byte count
    nbytes = int(st["d2h_bytes"])
    src = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    dst = hd.view(torch.uint8).reshape(-1)[:nbytes] if hd.numel() * 8 >= nbytes else \
        torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    ys = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dst.copy_(src, non_blocking=True)
        torch.cuda.synchronize()
        ys.append(time.perf_counter() - t0)
    plain_gbs = nbytes / min(ys) / 1e9
    del src
    # peak pool use against the batch size (offload on), beside the device
    # memory the same pass needs un-staged: sources, counts and offsets, all
    # coupled lists, the dedup workspace, the distinct set and the inverse
    curve = []
    for be in (batch // 4, batch, batch * 4, batch * 16):
        bufs = cusci.stream_buffers(sysd, s.dets, be, ucap, 0)
        bufs["hd"], bufs["hh"] = buffers["hd"], buffers["hh"]  # pinned sinks reused
        r = cusci.stream_gen_dedup(sysd, s.dets, s.eps, be, ucap, buffers=bufs)
        del bufs
        curve.append({"batch_entries": be, "pool_bytes": int(r[4]["pool_bytes"]),
                      "pool_peak_bytes": int(r[4]["pool_peak"]), "batches": int(r[4]["batches"]),
                      "ms": r[4]["batches_ms"] + r[4]["final_sort_ms"]})
        del r
        torch.cuda.empty_cache()
    W = sysd.W
    n_src, total_all, n_u = s.dets.shape[0], int(st["total"]), int(uniq.shape[0])
    unstaged = (n_src * 8 * W + 2 * (n_src + 1) * 8 + total_all * (8 * W + 8)
                + cusci.dedup_workspace(total_all, W, 2 * s.norb, s.n_alpha + s.n_beta)
                + n_u * 8 * W + total_all * 4)
    # Stage-3 reverse index of the host-resident coupled set against the device
    # distinct set, streamed back in batches
    total_e = st["total"]
    h_inv = torch.empty(total_e, dtype=torch.int32).pin_memory()
    rstatus = torch.zeros(1, dtype=torch.int32, device=dev)
    cusci.reverse_index_stream(uniq, hd[:total_e], batch=batch, host_out=h_inv, status=rstatus)
    rts = []
    for _ in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cusci.reverse_index_stream(uniq, hd[:total_e], batch=batch, host_out=h_inv,
                                   status=rstatus)
        rts.append(time.perf_counter() - t0)
    rt = min(rts)
    # the hashed form: a table of the distinct set built once, then probed by
    # every streamed batch (what a repeated Stage-3 query of one set costs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rtab = cusci.reverse_table(uniq, status=rstatus)
    torch.cuda.synchronize()
    t_build = time.perf_counter() - t0
    h_inv2 = torch.empty_like(h_inv).pin_memory()
    tts = []
    for _ in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cusci.reverse_index_stream(uniq, hd[:total_e], batch=batch, host_out=h_inv2,
                                   status=rstatus, table=rtab)
        tts.append(time.perf_counter() - t0)
    tt = min(tts)
    del rtab
    rev = {"entries_per_s": total_e / rt, "ms": rt * 1e3,
           "h2d_bytes": total_e * 8 * sysd.W, "d2h_bytes": total_e * 4,
           "transfer_gbs": total_e * (8 * sysd.W + 4) / rt / 1e9,
           "hashed": {"table_build_ms": t_build * 1e3, "ms": tt * 1e3,
                      "entries_per_s": total_e / tt,
                      "same_ids": bool(torch.equal(h_inv, h_inv2))},
           "status": int(rstatus.item())}
    hbm_peak, _ = _peaks()
    # W = 2: 16 + 8 written per entry, 16 read + 4 inverse-equivalent + 16 per distinct key
    alg = st["total"] * 48 + int(uniq.shape[0]) * 16
    return {"entries_per_s": st["total"] / t, "ms": t * 1e3, "entries": st["total"],
            "algorithmic_bytes": alg, "achieved_gbs": alg / t / 1e9,
            "frac_of_hbm": alg / t / 1e9 / hbm_peak,
            "unique": int(uniq.shape[0]), "batches": st["batches"],
            "batch_entries": batch, "pool_bytes": st["pool_bytes"],
            "pool_peak_bytes": st["pool_peak"], "batch_region_bytes": 2 * batch * 24,
            "coupled_set_bytes": st["total"] * 24, "d2h_bytes": st["d2h_bytes"],
            "d2h_gbs": st["d2h_bytes"] / t / 1e9, "plain_pinned_d2h_gbs": plain_gbs,
            "batches_ms": st["batches_ms"], "final_sort_ms": st["final_sort_ms"],
            "runs_ms": run_ms,
            "unique_capacity": ucap, "peak_vs_batch": curve, "unstaged_peak_bytes": unstaged,
            "pool_peak_vs_unstaged": st["pool_peak"] / unstaged,
            "reverse_index": rev,
            "workload": f"large: 120 spin orbitals (2 words), 10a+10b, {s.dets.shape[0]} sources, "
                        "eps 1e-6; host sources in, host coupled lists + device distinct set out; "
                        "then the reverse index of the host coupled set streamed back in"}


def run_batched(args, dev):
    """64 independent systems of uneven size (the batched workload; at
    --batch-scale 1, 1k-50k sources per system).  Systems are taken in order in
    waves of at most --batch-wave-entries coupled entries (the whole workload,
    ~6.4e9 entries, does not fit the device at once); every wave is one Batch:
    one persistent count launch, one persistent fill launch and one batched
    de-duplication of all its systems, autotuned (work-item size and grid) and
    replayed from a CUDA graph.  The time is the sum of the waves' replays."""
    import torch

    from paper_2604_15768_gb300 import cusci, synth
    t0 = time.perf_counter()
    systems = synth.batched_systems(64, scale=args.batch_scale)
    t_synth = time.perf_counter() - t0
    # exact entries of every system (one count pass each) to form the waves
    sizes = []
    for x in systems:
        sysd = cusci.System.of(x)
        sizes.append(int(cusci.count_coupled(sysd, cusci.dets_to_device(x.dets, dev),
                                             x.eps).sum().item()))
        del sysd
    waves, cur, acc = [], [], 0
    for k, m in enumerate(sizes):
        if cur and acc + m > args.batch_wave_entries:
            waves.append(cur)
            cur, acc = [], 0
        cur.append(k)
        acc += m
    if cur:
        waves.append(cur)
    hbm_peak, _ = _peaks()
    total_ms, total_entries, alg, uniq_total, launches, tuned = 0.0, 0, 0, 0, 0, []
    for wv in waves:
        ws_ = [systems[k] for k in wv]
        b = cusci.Batch(ws_, [x.dets for x in ws_], 1e-8, chunk=8)
        b.plan()
        (chunk, grid), _ = b.autotune(candidates=(1, 4, 16, 64), grids=(4, 8, 16), reps=1)
        b.capture()
        for _ in range(2):
            b.replay()
        torch.cuda.synchronize()
        l0 = cusci.kernel_launches()
        ts = []
        for _ in range(3):
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            b.replay()
            z.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(z))
        total_ms += float(np.median(ts))
        total_entries += b.total
        nus = b.n_unique.cpu().numpy()
        assert int(b.status.item()) == 0
        for j, x in enumerate(ws_):
            m = int(b.entry_begin[j + 1] - b.entry_begin[j])
            wbytes = 8 * x.W
            alg += m * (wbytes + 8) + m * (wbytes + 4) + int(nus[j]) * wbytes
        uniq_total += int(nus.sum())
        tuned.append({"systems": len(wv), "entries": b.total, "chunk": int(chunk),
                      "blocks_per_sm": int(grid), "ms": float(np.median(ts))})
        b.close()
        del b
        torch.cuda.empty_cache()
    return {"entries_per_s": total_entries / (total_ms * 1e-3), "ms": total_ms,
            "entries": total_entries, "algorithmic_bytes": alg,
            "achieved_gbs": alg / (total_ms * 1e-3) / 1e9,
            "frac_of_hbm": alg / (total_ms * 1e-3) / 1e9 / hbm_peak,
            "systems": len(systems), "sources": int(sum(x.dets.shape[0] for x in systems)),
            "waves": tuned, "unique_total": uniq_total, "synth_s": t_synth,
            "workload": f"64 systems, norb 10..50, 4..16 electrons, sources "
                        f"floor(logU(1e3,5e4) x {args.batch_scale}), eps 1e-8; waves of at most "
                        f"{args.batch_wave_entries:.3g} entries, each a graph replay of "
                        "count+scan+fill+batched dedup"}


REF_SOURCES = {"mid": 2000, "tiny": None, "large": 60}


def ref_sample(args):
    n = args.ref_sources if args.ref_sources is not None else REF_SOURCES[args.workload]
    return n


def run_cpu_baseline(args):
    from oracle import oracle as O
    from paper_2604_15768_gb300 import synth
    s = synth.config_system(args.workload, n_dets=ref_sample(args))
    osys = O.OracleSystem.of(s)
    t0 = time.perf_counter()
    counts = osys.count(s.dets, s.eps)
    off, td, hv = osys.gen(s.dets, s.eps, counts)
    O.dedup(td)
    t = time.perf_counter() - t0
    return {"value": int(off[-1]) / t, "unit": UNIT, "cores": O.threads(), "kind": "oracle",
            "sample": f"first {s.dets.shape[0]} sources of the {args.workload} workload "
                      f"(count+gen+dedup, {int(off[-1])} entries, {t:.1f} s)"}


def run_profile(args):
    """Profiling driver (for ncu): count -> scan -> fill -> dedup of the first
    ``--profile-sources`` sources of the workload through the public API, the
    warm-up steps and then ``--steps`` steps, with no extra legs.  Prints one
    JSON line with the sizes and CUDA-event times; not a benchmark line."""
    import torch

    from paper_2604_15768_gb300 import cusci, synth

    torch.cuda.set_device(0)
    s = synth.config_system(args.workload, n_dets=args.profile_sources)
    sysd = cusci.System.of(s)
    n, W = s.dets.shape
    d_src = cusci.dets_to_device(s.dets)
    n_bits, n_ones = 2 * s.norb, s.n_alpha + s.n_beta
    times = []
    for it in range(args.warmup + args.steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        off, od, oh, st = cusci.coupled(sysd, d_src, s.eps)
        u, inv, nu = cusci.dedup(od, n_bits, n_ones, sync=False)
        b.record()
        torch.cuda.synchronize()
        if it >= args.warmup:
            times.append(a.elapsed_time(b))
        total = od.shape[0]
        n_unique = int(nu.item())
        del off, od, oh, st, u, inv, nu
    print(json.dumps({"profile": WORKLOADS[args.workload].format(n=n), "entries": total,
                      "unique": n_unique, "ms": times}), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mid", choices=sorted(WORKLOADS),
                    help="workload of the timed step (the metric is quoted on 'mid')")
    ap.add_argument("--sources", type=int, default=None,
                    help="number of sources (default: the workload's own)")
    ap.add_argument("--energy-sources", type=int, default=200_000)
    ap.add_argument("--ref-sources", type=int, default=None,
                    help="sources of the CPU-oracle sample (default per workload)")
    ap.add_argument("--no-e2e", dest="e2e", action="store_false")
    ap.add_argument("--no-energy", dest="energy", action="store_false")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-stream", dest="stream", action="store_false")
    ap.add_argument("--no-batched", dest="batched", action="store_false")
    ap.add_argument("--no-ranks", dest="ranks", action="store_false")
    ap.add_argument("--stream-sources", type=int, default=20_000)
    ap.add_argument("--stream-batch", type=int, default=16_000_000)
    ap.add_argument("--stream-unique-cap", type=int, default=0,
                    help="distinct-set capacity of the streaming leg (0: measured + 10%%)")
    ap.add_argument("--batch-scale", type=float, default=1.0)
    ap.add_argument("--batch-wave-entries", type=float, default=1.2e9)
    ap.add_argument("--profile-sources", type=int, default=None,
                    help="profiling driver: count/scan/fill/dedup of this many sources only")
    ap.add_argument("--profile-batched", action="store_true",
                    help="profiling driver: the batched leg alone (at --batch-scale)")
    args = ap.parse_args(argv)
    if args.profile_sources:
        return run_profile(args)
    if args.profile_batched:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps({"profile": "batched", "batched": run_batched(args, torch.device("cuda:0"))}),
              flush=True)
        return 0
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
